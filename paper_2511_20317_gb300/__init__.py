"""GB300 (sm_103a) walker library for ternary flip-graph search of matrix
multiplication schemes (arXiv 2511.20317).

* ``paper_2511_20317_gb300.tfg``: ctypes binding of ``libtfg.so`` (C ABI in
  ``include/tfg.h``): device walkers, host scheme checks and meta operators.
* ``paper_2511_20317_gb300.workloads``: synthetic start schemes and the
  populations of the measured workloads.
* ``paper_2511_20317_gb300._build``: nvcc build of ``libtfg.so``.
"""
__all__ = ["tfg", "workloads"]
