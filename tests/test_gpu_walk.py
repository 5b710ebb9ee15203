"""GPU parity: the CUDA walkers (through the C ABI) against the CPU oracle,
bit-exact on every compared walker's slots, best scheme, counters and
trajectory digest."""
import os

import numpy as np
import pytest

import oracle
from paper_2511_20317_gb300 import tfg
from paper_2511_20317_gb300.tfg import WALKER_INFO_DTYPE, term_len
from paper_2511_20317_gb300.workloads import golden_dir, naive_start, read_scheme, workload_mixed

pytestmark = pytest.mark.gpu

THREADS = len(os.sched_getaffinity(0))
FIELDS = ["r", "best_r", "t", "plateau", "best_t", "digest", "accepted", "rejected", "nocand", "drops",
          "merges", "plus", "reductions"]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2511_20317_gb300 import _build
    _build.build()
    tfg.lib()
    torch.cuda.set_device(0)


def gpu_walkers(fmt, mode, start, nw, seed, steps, chunks=1, **params):
    p = tfg.tfg_default_params(**params)
    W = tfg.Walkers([(fmt, mode, start, nw)], seed=seed, params=p)
    for c in range(chunks):
        W.walk(steps // chunks + (steps % chunks if c == chunks - 1 else 0))
    W.sync()
    return W


def assert_parity(info, slots, best, ref, ref_rows, label=""):
    """info/slots/best: GPU rows; ref: oracle.Walkers; ref_rows: oracle indices."""
    for a, w in enumerate(ref_rows):
        oi = ref.info[w]
        for f in FIELDS:
            assert info[f][a] == oi[f], f"{label} walker row {a}: {f} gpu={info[f][a]} oracle={oi[f]}"
        r, br = oi["r"], oi["best_r"]
        assert np.array_equal(slots[a, :r], ref.slots[w, :r]), f"{label} walker row {a}: slots differ"
        assert np.array_equal(best[a, :br], ref.best[w, :br]), f"{label} walker row {a}: best differs"


def test_philox_device_matches_oracle():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, size=(257, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key = (0xA4093822, 0x299F31D0)
    got = tfg.tfg_philox_device(ctr.reshape(-1), *key).reshape(-1, 4)
    for k in range(ctr.shape[0]):
        assert list(got[k]) == list(oracle.philox4x32_10(ctr[k], key))
    kat = tfg.tfg_philox_device(np.array([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], np.uint32),
                                0xA4093822, 0x299F31D0)
    assert list(kat) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


@pytest.mark.parametrize("mode", [tfg.TFG_MODE_ZT, tfg.TFG_MODE_Z2])
@pytest.mark.parametrize("lanes", [1, 4, 8, 16, 32])
@pytest.mark.parametrize("fmt,L,steps,nw", [((2, 2, 2), 200, 6000, 300), ((3, 3, 3), 600, 4000, 200),
                                            ((2, 3, 4), 400, 3000, 130)])
def test_parity_small_all_mappings(fmt, L, steps, nw, lanes, mode):
    seed = 17
    start = naive_start(*fmt)
    W = gpu_walkers(fmt, mode, start, nw, seed, steps, chunks=3, plateau_len=L, mapping=lanes)
    assert W.pop[0]["lanes"] == lanes
    # thread per walker: capacity 32 with factors of at most 9 coefficients is the bit-sliced kernel
    assert W.pop[0]["slice_len"] == (9 if lanes == 1 and fmt == (3, 3, 3) else 0)
    assert W.pop[0]["square"] == (1 if lanes == 1 and fmt == (3, 3, 3) else 0)
    info, slots, best = W.read_walkers(0, nw)
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=seed, mode=mode, plateau_len=L).walk(steps, THREADS)
    assert (ref.info["plus"] > 0).any() and (ref.info["merges"] > 0).any()
    assert_parity(info, slots, best, ref, range(nw), f"{fmt} G={lanes} mode={mode}")
    assert W.verify_all() == 0
    W.close()


@pytest.mark.parametrize("mode", [tfg.TFG_MODE_ZT, tfg.TFG_MODE_Z2])
@pytest.mark.parametrize("fmt", [(2, 3, 3), (3, 2, 3), (3, 3, 2), (1, 3, 3)])
def test_bit_sliced_kernel_uneven_factors(fmt, mode):
    """The bit-sliced thread-per-walker kernel on formats whose factors are
    shorter than the slice length (6 or 3 of 9 coefficients, factor offsets
    that are not multiples of 9); the slack lifts the capacity to 32."""
    start = naive_start(*fmt)
    if mode == tfg.TFG_MODE_Z2:
        start = np.abs(start).astype(np.int8)
    nw, steps, L = 160, 3000, 150
    slack = 32 - start.shape[0]
    W = gpu_walkers(fmt, mode, start, nw, 21, steps, chunks=2, plateau_len=L, r_slack=slack, mapping=1)
    assert W.pop[0]["slice_len"] == 9 and W.pop[0]["square"] == 0 and W.pop[0]["r_max"] == 32
    info, slots, best = W.read_walkers(0, nw)
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=21, mode=mode, plateau_len=L, r_slack=slack).walk(steps, THREADS)
    assert (ref.info["accepted"] > 0).all() and (ref.info["plus"] > 0).any()
    assert_parity(info, slots, best, ref, range(nw), f"sliced {fmt} mode={mode}")
    assert W.verify_all() == 0
    W.close()


def test_parity_222_full_workload_all_walkers():
    """(2,2,2) Z_T from the naive rank-8 scheme: 1024 walkers x 1e5 steps,
    plateau 1e4; every walker replayed by the oracle."""
    fmt, nw, steps, L = (2, 2, 2), 1024, 100_000, 10_000
    start = naive_start(*fmt)
    W = gpu_walkers(fmt, tfg.TFG_MODE_ZT, start, nw, 0, steps, plateau_len=L)
    info, slots, best = W.read_walkers(0, nw)
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=0, plateau_len=L).walk(steps, THREADS)
    assert_parity(info, slots, best, ref, range(nw), "222-full")
    assert W.verify_all() == 0
    scheme, rank, walker = W.collect_best(0)
    assert rank == info["best_r"].min() and walker == int(np.argmin(info["best_r"]))
    assert tfg.tfg_verify(fmt, scheme) and oracle.brent_valid(fmt, scheme)
    W.close()


@pytest.mark.parametrize("mode,seed", [(tfg.TFG_MODE_ZT, 0), (tfg.TFG_MODE_Z2, 1)])
def test_parity_333_full_population_sampled(mode, seed):
    """(3,3,3) from the naive rank-27 scheme, 65536 walkers, plateau 5e4; the
    GPU runs the whole population, the oracle replays walkers 256*k."""
    fmt, nw, steps, L = (3, 3, 3), 65536, 200_000, 50_000
    start = naive_start(*fmt)
    W = gpu_walkers(fmt, mode, start, nw, seed, steps, chunks=2, plateau_len=L)
    sample = np.arange(0, nw, 256)
    infos, slots, bests = [], [], []
    for w in sample:
        i, s, b = W.read_walkers(int(w), 1)
        infos.append(i); slots.append(s); bests.append(b)
    info = np.concatenate(infos)
    ref = oracle.Walkers(fmt, start, sample, seed=seed, mode=mode, plateau_len=L).walk(steps, THREADS)
    assert_parity(info, np.concatenate(slots), np.concatenate(bests), ref, range(sample.size), f"333 mode={mode}")
    assert W.verify_all() == 0
    W.close()


def test_chunking_and_checkpoint_resume():
    fmt, nw, L = (3, 3, 3), 512, 700
    start = naive_start(*fmt)
    p = tfg.tfg_default_params(plateau_len=L)
    A = tfg.Walkers([(fmt, 0, start, nw)], seed=3, params=p)
    A.walk(2500).sync()
    ck = A.checkpoint()
    A.walk(2501).sync()
    ia, sa, ba = A.read_walkers(0, nw)
    B = tfg.Walkers([(fmt, 0, start, nw)], seed=3, params=p)
    B.restore(ck)
    B.walk(1000).walk(1501).sync()
    ib, sb, bb = B.read_walkers(0, nw)
    assert np.array_equal(ia, ib) and np.array_equal(sa, sb) and np.array_equal(ba, bb)
    C = tfg.Walkers([(fmt, 0, start, nw)], seed=3, params=p)
    C.walk(5001).sync()
    ic, sc, bc = C.read_walkers(0, nw)
    assert np.array_equal(ia, ic) and np.array_equal(sa, sc)


def test_shards_equal_single_run():
    """Walker ids are global (walker_id_base): two half populations reproduce one
    whole population, as a two-GPU split would."""
    fmt, nw, L, steps = (2, 3, 4), 600, 500, 3000
    start = naive_start(*fmt)
    whole = gpu_walkers(fmt, 0, start, nw, 8, steps, plateau_len=L)
    iw, sw, bw = whole.read_walkers(0, nw)
    lo = gpu_walkers(fmt, 0, start, 250, 8, steps, plateau_len=L, walker_id_base=0)
    hi = gpu_walkers(fmt, 0, start, 350, 8, steps, plateau_len=L, walker_id_base=250)
    i1, s1, b1 = lo.read_walkers(0, 250)
    i2, s2, b2 = hi.read_walkers(0, 350)
    assert np.array_equal(np.concatenate([i1, i2]), iw)
    assert np.array_equal(np.concatenate([s1, s2]), sw) and np.array_equal(np.concatenate([b1, b2]), bw)


def test_mixed_formats_one_context():
    """Five formats of the mixed workload (naive starts) in one context; each
    population checked against the oracle with its global walker ids."""
    wl = workload_mixed(total=1040)
    pops = [(p.fmt, 0, p.start_scheme(), p.walkers) for p in wl.populations]
    L, steps, seed = 800, 2000, 0
    W = tfg.Walkers(pops, seed=seed, params=tfg.tfg_default_params(plateau_len=L))
    W.walk(steps).sync()
    for f, pop in enumerate(W.pop):
        take = np.linspace(0, pop["walkers"] - 1, 12).astype(int)
        rows = [W.read_walkers(pop["first"] + int(w), 1) for w in take]
        info = np.concatenate([x[0] for x in rows])
        ids = pop["first"] + take
        assert (info["walker_id"] == ids).all()
        ref = oracle.Walkers(pop["fmt"], wl.populations[f].start_scheme(), ids, seed=seed,
                             plateau_len=L).walk(steps, THREADS)
        assert_parity(info, np.concatenate([x[1] for x in rows]), np.concatenate([x[2] for x in rows]), ref,
                      range(len(take)), f"mixed {pop['fmt']}")
    assert W.verify_all() == 0


def test_mixed_full_population_sampled():
    """The mixed workload at its full size (262144 walkers in five populations,
    one context, one graph launch per chunk): 16 walkers per format, spread over
    each population, replayed by the oracle with their global walker ids."""
    wl = workload_mixed()
    pops = [(p.fmt, 0, p.start_scheme(), p.walkers) for p in wl.populations]
    assert [p[3] for p in pops] == [20165, 40330, 40330, 80660, 80659]
    L, steps, seed = 5000, 20000, 0
    W = tfg.Walkers(pops, seed=seed, params=tfg.tfg_default_params(plateau_len=L))
    W.walk(steps // 2).walk(steps - steps // 2).sync()
    for f, pop in enumerate(W.pop):
        take = np.linspace(0, pop["walkers"] - 1, 16).astype(int)
        rows = [W.read_walkers(pop["first"] + int(w), 1) for w in take]
        info = np.concatenate([x[0] for x in rows])
        ids = pop["first"] + take
        ref = oracle.Walkers(pop["fmt"], wl.populations[f].start_scheme(), ids, seed=seed,
                             plateau_len=L).walk(steps, THREADS)
        assert_parity(info, np.concatenate([x[1] for x in rows]), np.concatenate([x[2] for x in rows]), ref,
                      range(len(take)), f"mixed full {pop['fmt']}")
    assert W.verify_all() == 0
    W.close()


@pytest.mark.parametrize("fmt,block", [((2, 4, 5), 96), ((3, 4, 5), 128), ((4, 4, 4), 128), ((4, 4, 5), 160)])
def test_walkers_per_block_choices_are_bit_exact(fmt, block):
    """The other compiled walkers-per-block choices of the thread-per-walker
    kernels (selected through tfg_params.block_threads; the autotuner times them
    all): capacities 48, 64, 72 and 88 at 96, 128, 128 and 160 threads per block."""
    start = naive_start(*fmt)
    nw, steps, L = 700, 1500, 300
    W = gpu_walkers(fmt, 0, start, nw, 31, steps, chunks=2, plateau_len=L, block_threads=block)
    assert W.pop[0]["lanes"] == 1 and W.pop[0]["block_threads"] == block
    assert W.pop[0]["grid"] == (nw + block - 1) // block
    info, slots, best = W.read_walkers(0, nw)
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=31, plateau_len=L).walk(steps, THREADS)
    assert (ref.info["accepted"] > 0).all() and (ref.info["plus"] > 0).any()
    assert_parity(info, slots, best, ref, range(nw), f"{fmt} block {block}")
    assert W.verify_all() == 0
    W.close()


def test_large_formats_full_population_sampled():
    """The large-format workload at its full size: (4,5,12), (5,6,10), (6,7,9) from the
    meta-operator starts, 131072 walkers each, one forked graph launch per chunk (the
    bench's configuration), 50000 steps; 4 walkers per format, spread over each
    population, replayed by the oracle with their global walker ids."""
    from paper_2511_20317_gb300 import starts
    pops = starts.large_populations(131072)
    L, steps, seed = 50_000, 50_000, 0
    W = tfg.Walkers(pops, seed=seed, params=tfg.tfg_default_params(plateau_len=L, use_graph=2))
    W.walk(steps // 2).walk(steps - steps // 2).sync()
    for f, pop in enumerate(W.pop):
        assert pop["slots_per_lane"] == 0, "warp-per-walker kernel expected"
        take = np.linspace(0, pop["walkers"] - 1, 4).astype(int)
        rows = [W.read_walkers(pop["first"] + int(w), 1) for w in take]
        info = np.concatenate([x[0] for x in rows])
        ids = pop["first"] + take
        ref = oracle.Walkers(pop["fmt"], pops[f][2], ids, seed=seed, plateau_len=L).walk(steps, THREADS)
        assert (ref.info["accepted"] > 0).all()
        assert_parity(info, np.concatenate([x[1] for x in rows]), np.concatenate([x[2] for x in rows]), ref,
                      range(len(take)), f"large full {pop['fmt']}")
    W.close()


def test_large_formats_million_step_prefix():
    """The large-format trajectories over a 1e6-step prefix: 4 walkers per format
    at the global ids they have in the full 131072-walker populations (the middle
    of each population), in one context per format with walker_id_base set to
    those ids (a trajectory depends only on seed, id and step, and the kernel
    variant only on the format and capacity, so these are the full run's
    trajectories), the three formats on their own streams; replayed by the oracle."""
    import torch
    from paper_2511_20317_gb300 import starts
    pops = starts.large_populations(131072)
    L, steps, seed, nw = 50_000, 1_000_000, 0, 4
    ctxs, ids = [], []
    for f, (fmt, mode, start, total) in enumerate(pops):
        base = f * total + total // 2
        st = torch.cuda.Stream()
        W = tfg.Walkers([(fmt, mode, start, nw)], seed=seed, stream=st,
                        params=tfg.tfg_default_params(plateau_len=L, walker_id_base=base))
        assert W.pop[0]["slots_per_lane"] == 0, "warp-per-walker kernel expected"
        ctxs.append(W)
        ids.append(base + np.arange(nw))
    for _ in range(steps // 100_000):
        for W in ctxs:
            W.walk(100_000)
    for W in ctxs:
        W.sync()
    refs = [oracle.Walkers(p[0], p[2], i, seed=seed, plateau_len=L) for p, i in zip(pops, ids)]
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(len(refs)) as ex:   # all twelve walkers at once over the host cores
        list(ex.map(lambda rf: rf.walk(steps, max(1, THREADS // len(refs))), refs))
    for W, ref, (fmt, *_rest) in zip(ctxs, refs, pops):
        info, slots, best = W.read_walkers(0, nw)
        assert (ref.info["accepted"] > 0).all() and (info["t"] == steps).all()
        assert_parity(info, slots, best, ref, range(nw), f"large 1e6 prefix {fmt}")
        W.close()


def test_start_from_paper_scheme_and_edge_formats():
    """Start from the (2,2,3:11) example of Section 3.1.1; and the degenerate
    formats (1,1,1) (rank 1: no candidate ever) and (1,2,1)."""
    fmt, s = read_scheme(os.path.join(golden_dir(), "paper_2x2x3_r11.txt"))
    for (f, st, nw) in [(fmt, s, 96), ((1, 1, 1), naive_start(1, 1, 1), 40), ((1, 2, 1), naive_start(1, 2, 1), 40),
                        ((1, 1, 5), naive_start(1, 1, 5), 33)]:
        W = gpu_walkers(f, 0, st, nw, 2, 2000, plateau_len=100)
        info, slots, best = W.read_walkers(0, nw)
        ref = oracle.Walkers(f, st, np.arange(nw), seed=2, plateau_len=100).walk(2000, THREADS)
        assert_parity(info, slots, best, ref, range(nw), f"edge {f}")
        if f == (1, 1, 1):
            assert (info["nocand"] == 2000).all()
        assert W.verify_all() == 0


def _start_4_5_12():
    fmt_s, S = read_scheme(os.path.join(golden_dir(), "strassen_2x2x2_r7.txt"))
    f1, s1 = tfg.tfg_extend(fmt_s, S, 2)
    f2, s2 = tfg.tfg_double(f1, s1, 2)
    f3, s3 = tfg.tfg_product(fmt_s, S, f2, s2)
    f4, s4 = tfg.tfg_extend(f3, s3, 1)
    assert f4 == (4, 5, 12) and s4.shape[0] == 202
    return f4, s4


@pytest.mark.parametrize("mode", [tfg.TFG_MODE_ZT, tfg.TFG_MODE_Z2])
@pytest.mark.parametrize("case", ["4x5x5", "4x5x12", "8x8x1", "1x8x8", "6x7x9", "8x8x8"])
def test_wide_terms_parity(case, mode):
    """Terms longer than 64 coefficients (factor-aligned words, shared-memory
    signature search): naive (4,5,5) and (6,7,9), the meta-operator (4,5,12)
    start of rank 202, and factors of exactly 64 coefficients."""
    if case == "4x5x12":
        fmt, start = _start_4_5_12()
        nw, steps, L = 40, 1500, 300
    else:
        fmt = tuple(int(x) for x in case.split("x"))
        start = naive_start(*fmt)
        nw, steps, L = {"4x5x5": (64, 3000, 300), "8x8x1": (64, 2000, 200), "1x8x8": (64, 2000, 200),
                        "6x7x9": (12, 400, 100), "8x8x8": (6, 300, 60)}[case]
    if case in ("6x7x9", "8x8x8") and mode == tfg.TFG_MODE_Z2:
        pytest.skip("one mode suffices at ranks 378 and 512")
    if mode == tfg.TFG_MODE_Z2:
        start = np.abs(start).astype(np.int8)   # a Z_T scheme read mod 2
    W = gpu_walkers(fmt, mode, start, nw, 4, steps, chunks=2, plateau_len=L)
    assert W.pop[0]["slots_per_lane"] == 0, "wide-term kernel expected"
    info, slots, best = W.read_walkers(0, nw)
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=4, mode=mode, plateau_len=L).walk(steps, THREADS)
    if case in ("4x5x5", "8x8x1"):
        assert (ref.info["merges"] > 0).any() and (ref.info["plus"] > 0).any()
    assert_parity(info, slots, best, ref, range(nw), f"wide {fmt} mode={mode}")
    assert W.verify_all() == 0
    W.close()


@pytest.mark.parametrize("policy", [0, 1, 2])
@pytest.mark.parametrize("mode", [tfg.TFG_MODE_ZT, tfg.TFG_MODE_Z2])
@pytest.mark.parametrize("case", ["9x1x8", "1x9x9", "11x11x1", "9x8x2", "2x9x8"])
def test_two_word_factor_parity(case, mode, policy):
    """Factors longer than 64 coefficients (two 64-bit words per factor and
    sign): the long factor in each of the u, v and w positions; shared-memory
    terms (ranks 72-121) and HBM terms (rank 144); the three walk policies."""
    fmt = tuple(int(x) for x in case.split("x"))
    if policy and case not in ("9x1x8", "9x8x2"):
        pytest.skip("walk policies 1 and 2 on one shared-memory and one HBM case")
    start = naive_start(*fmt)
    if mode == tfg.TFG_MODE_Z2:
        start = np.abs(start).astype(np.int8)
    big = fmt[0] * fmt[1] * fmt[2] > 128
    nw, steps, L = (16, 3000, 200) if big else (32, 1500, 150)
    kw = dict(plateau_len=L, walk_policy=policy)
    if policy == 1:
        kw["expand_thresh"] = 1 << 27
    W = gpu_walkers(fmt, mode, start, nw, 6, steps, chunks=2, **kw)
    assert W.pop[0]["slots_per_lane"] == 0, "wide-term kernel expected"
    info, slots, best = W.read_walkers(0, nw)
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=6, mode=mode, plateau_len=L, policy=policy,
                         expand_thresh=kw.get("expand_thresh", 0)).walk(steps, THREADS)
    if policy == 0 and not big:
        assert (ref.info["merges"] > 0).any() and (ref.info["plus"] > 0).any()
    assert_parity(info, slots, best, ref, range(nw), f"two-word {fmt} mode={mode} policy={policy}")
    assert W.verify_all() == 0
    W.close()


def test_graph_launch_equals_stream_launch_and_autotune_restores_state():
    """The mixed populations run as one captured graph (forked: one concurrent
    branch per format) or as plain launches on one stream: identical results.  The autotuner's
    trial runs leave no trace in the walkers' state."""
    wl = workload_mixed(total=6000)
    pops = [(p.fmt, 0, p.start_scheme(), p.walkers) for p in wl.populations]
    A = tfg.Walkers(pops, seed=2, params=tfg.tfg_default_params(plateau_len=300, use_graph=2))
    B = tfg.Walkers(pops, seed=2, params=tfg.tfg_default_params(plateau_len=300, use_graph=0))
    A.walk(700)
    B.walk(700)
    lanes = A.autotune(trial_steps=150, trial_walkers=900)
    assert len(lanes) == len(pops) and all(g in (1, 4, 8, 16, 32) for g in lanes)
    A.walk(800).walk(500)
    B.walk(1300)
    for pop in A.pop:
        ia, sa, ba = A.read_walkers(pop["first"], pop["walkers"])
        ib, sb, bb = B.read_walkers(pop["first"], pop["walkers"])
        assert np.array_equal(ia, ib) and np.array_equal(sa, sb) and np.array_equal(ba, bb), pop["fmt"]
    assert A.verify_all() == 0


def _best_region(W, f):
    """Where population f's best slots sit inside a checkpoint blob: the blob
    starts at the first walker record; records, live slots, best slots and the
    packed start follow one another, each padded to 256 bytes.  Terms of at
    most 64 coefficients concatenate u|v|w in one word per sign (32-bit words
    up to 32 coefficients); longer ones hold factor f in 64-bit word f."""
    p = W.pop[f]
    assert f == 0
    fmt, mode, n, R = p["fmt"], p["mode"], p["walkers"], p["r_max"]
    m, nn, pp = fmt
    lt = term_len(fmt)
    if lt <= 64:
        wb, tw = (4 if lt <= 32 else 8), 1
        coef_bit = np.arange(lt)
    else:
        wb, tw = 8, 3
        lens = [m * nn, nn * pp, pp * m]
        coef_bit = np.concatenate([64 * x + np.arange(lens[x]) for x in range(3)])
    nws = (2 if mode == tfg.TFG_MODE_ZT else 1) * tw
    per = R * nws * wb
    up = lambda x: (x + 255) // 256 * 256
    off_best = up(n * WALKER_INFO_DTYPE.itemsize) + up(n * per)
    return off_best, per, wb, tw, nws, coef_bit


@pytest.mark.parametrize("which", ["333zt", "333z2", "4512zt", "569z2"])
def test_verify_all_flags_exactly_the_corrupted_walkers(which):
    """Eq. (1) on the device: change one coefficient of the best scheme of some
    walkers (through a checkpoint blob) and exactly those walkers fail."""
    from paper_2511_20317_gb300 import starts
    if which == "333zt":
        fmt, mode, start = (3, 3, 3), tfg.TFG_MODE_ZT, naive_start(3, 3, 3)
    elif which == "333z2":
        fmt, mode, start = (3, 3, 3), tfg.TFG_MODE_Z2, naive_start(3, 3, 3)
    elif which == "4512zt":
        (fmt, start), mode = starts.start_4_5_12(), tfg.TFG_MODE_ZT
    else:
        fmt, mode, start = (5, 6, 9), tfg.TFG_MODE_Z2, naive_start(5, 6, 9)
    n = 48
    W = tfg.Walkers([(fmt, mode, start, n)], seed=3, params=tfg.tfg_default_params(plateau_len=400))
    W.walk(300).sync()
    assert W.verify_all() == 0
    info, _, best = W.read_walkers(0, n, slots=False)
    blob = np.frombuffer(W.checkpoint(), dtype=np.uint8).copy()
    off, per, wb, tw, nws, coef_bit = _best_region(W, 0)
    words = blob[off: off + n * per].view(np.uint32 if wb == 4 else np.uint64).reshape(n, -1, nws)
    # the located region decodes to the walkers' best schemes
    lt = term_len(fmt)
    bits = wb * 8
    for w in (0, n - 1):
        r = int(info["best_r"][w])
        e = coef_bit
        ww = words[w][:r]                                  # [r, nws]
        sh = (e % bits).astype(words.dtype)
        pos = (ww[:, e // bits] >> sh) & 1
        neg = ((ww[:, tw + e // bits] >> sh) & 1) if nws > tw else 0 * pos
        assert np.array_equal(pos.astype(np.int8) - neg.astype(np.int8), best[w, :r])
    bad = [1, 7, 30]
    rng = np.random.default_rng(5)
    for w in bad:
        term = int(rng.integers(info["best_r"][w]))
        coef = int(coef_bit[int(rng.integers(lt))])
        words[w, term, coef // bits] ^= words.dtype.type(1) << words.dtype.type(coef % bits)   # +1 bit toggled
        if nws > tw:
            words[w, term, tw + coef // bits] &= ~(words.dtype.type(1) << words.dtype.type(coef % bits))
    W.restore(blob.tobytes())
    assert W.verify_all() == len(bad)
    W.close()


@pytest.mark.parametrize("graph", [0, 1, 2])
def test_empty_populations_and_zero_steps(graph):
    """Populations of zero walkers are carried through every call: walks skip
    them (also inside a captured graph), statistics and checks ignore them,
    collecting their best scheme is an error; zero-step walks change nothing."""
    fmt = (2, 2, 2)
    p = tfg.tfg_default_params(plateau_len=100, use_graph=graph)
    W = tfg.Walkers([((3, 3, 3), 0, naive_start(3, 3, 3), 0), (fmt, 0, naive_start(*fmt), 100)], seed=5, params=p)
    before = W.checkpoint()
    W.walk(0).sync()
    assert W.checkpoint() == before
    W.walk(500).sync()
    assert W.verify_all() == 0
    with pytest.raises(tfg.TfgError) as e:
        W.collect_best(0)
    assert e.value.code == tfg.TFG_EINVAL
    scheme, rank, walker = W.collect_best(1)
    assert tfg.tfg_verify(fmt, scheme) and rank == scheme.shape[0]
    info, slots, best = W.read_walkers(W.pop[1]["first"], 100)
    ref = oracle.Walkers(fmt, naive_start(*fmt), np.arange(100), seed=5, plateau_len=100).walk(500, THREADS)
    assert_parity(info, slots, best, ref, range(100), f"empty+222 graph={graph}")
    W.close()
    E = tfg.Walkers([((3, 3, 3), 0, naive_start(3, 3, 3), 0)], seed=5, params=p)
    E.walk(10).sync()
    assert E.verify_all() == 0
    E.close()


@pytest.mark.parametrize("mode", [tfg.TFG_MODE_ZT, tfg.TFG_MODE_Z2])
@pytest.mark.parametrize("fmt,lanes,nw", [((2, 2, 2), 1, 200), ((3, 3, 3), 1, 150), ((2, 3, 4), 8, 100),
                                          ((3, 3, 3), 32, 64), ((4, 5, 5), 32, 40), ((6, 7, 9), 32, 8)])
def test_algorithm1_policy_parity(fmt, lanes, nw, mode):
    """Walk policy 1 (Algorithm 1 expansions, plus or split) on the thread-per-walker,
    lane-group and wide-term kernels against the oracle."""
    if fmt == (6, 7, 9) and mode == tfg.TFG_MODE_Z2:
        pytest.skip("one mode suffices at rank 378")
    start = naive_start(*fmt)
    steps, slack, thr = (1500, 10, int(0.03 * 2**32)) if fmt != (6, 7, 9) else (300, 8, int(0.05 * 2**32))
    if fmt == (3, 3, 3) and lanes == 1:
        slack = 5                      # capacity 32: the largest 32-bit thread-per-walker variant
    W = gpu_walkers(fmt, mode, start, nw, 9, steps, chunks=2, plateau_len=10**6, r_slack=slack, walk_policy=1,
                    expand_thresh=thr, mapping=lanes)
    info, slots, best = W.read_walkers(0, nw)
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=9, mode=mode, plateau_len=10**6, r_slack=slack, policy=1,
                         expand_thresh=thr).walk(steps, THREADS)
    assert (ref.info["plus"] > 0).any()
    assert_parity(info, slots, best, ref, range(nw), f"policy 1 {fmt} G={lanes} mode={mode}")
    assert W.verify_all() == 0
    W.close()


def test_window_mode_rejects_policy1():
    W = tfg.Walkers([((3, 3, 3), 0, naive_start(3, 3, 3), 32)], seed=1,
                    params=tfg.tfg_default_params(walk_policy=1, expand_thresh=1000))
    with pytest.raises(tfg.TfgError) as e:
        W.walk_window(1, policy=0)
    assert e.value.code == tfg.TFG_EINVAL
    W.close()


def test_reseed_continues_the_walkers_streams():
    """tfg_reseed replaces a block of walkers by a new scheme: their records restart
    at the prepared rank while the step count, counters and digest go on, so they
    walk on exactly like oracle walkers started from that scheme with those
    records; the other walkers are untouched."""
    fmt, n, L, slack = (2, 3, 3), 64, 300, 4
    start = naive_start(*fmt)
    A = gpu_walkers(fmt, 0, start, n, 6, 1000, plateau_len=L, r_slack=slack)
    B = gpu_walkers(fmt, 0, start, n, 6, 1000, plateau_len=L, r_slack=slack)
    R = A.pop[0]["r_max"]
    S = oracle.Walkers(fmt, start, [999], seed=1, plateau_len=L).walk(3000).scheme(0)   # a walked state
    prepared = oracle.prepare_start(fmt, S)
    A.reseed(10, 20, S)
    info0, _, _ = A.read_walkers(10, 20, slots=False, best=False)
    r0 = prepared.shape[0]
    assert (info0["r"] == r0).all() and (info0["best_r"] == r0).all()
    assert (info0["plateau"] == 0).all() and (info0["best_t"] == info0["t"]).all() and (info0["t"] == 1000).all()
    A.walk(700).sync()
    B.walk(700).sync()
    ia, sa, ba = A.read_walkers(0, n)
    ib, sb, bb = B.read_walkers(0, n)
    keep = np.r_[0:10, 30:n]
    assert np.array_equal(ia[keep], ib[keep]) and np.array_equal(sa[keep], sb[keep]) and np.array_equal(ba[keep], bb[keep])
    ref = oracle.Walkers(fmt, S, np.arange(10, 30), seed=6, plateau_len=L, r_slack=R - r0)
    assert ref.r_max == R
    for f in ["t", "plateau", "best_t", "digest", "accepted", "rejected", "nocand", "drops", "merges", "plus",
              "reductions"]:
        ref.info[f] = info0[f]
    ref.walk(700, THREADS)
    assert_parity(ia[10:30], sa[10:30], ba[10:30], ref, range(20), "reseeded")
    # errors: a range outside one population, a scheme violating Eq. (1), a rank above r_max
    with pytest.raises(tfg.TfgError) as e:
        A.reseed(60, 10, S)
    assert e.value.code == tfg.TFG_EINVAL
    bad = S.copy()
    bad[0, 0] = 0 if bad[0, 0] else 1
    with pytest.raises(tfg.TfgError) as e:
        A.reseed(0, 4, bad)
    assert e.value.code == tfg.TFG_ESCHEME
    grown = oracle.Walkers(fmt, start, np.arange(8), seed=2, r_slack=12, policy=1).walk(200)   # expansions
    big = next(grown.scheme(w) for w in range(8) if oracle.prepare_start(fmt, grown.scheme(w)).shape[0] > R)
    with pytest.raises(tfg.TfgError) as e:
        A.reseed(0, 4, big)
    assert e.value.code == tfg.TFG_ENOSPC
    A.close()
    B.close()


@pytest.mark.parametrize("mode", [tfg.TFG_MODE_ZT, tfg.TFG_MODE_Z2])
@pytest.mark.parametrize("fmt,lanes,nw", [((3, 3, 3), 1, 150), ((2, 3, 4), 8, 100), ((3, 3, 3), 32, 64),
                                          ((4, 5, 5), 32, 40), ((6, 7, 9), 32, 8)])
def test_complexity_policy_parity(fmt, lanes, nw, mode):
    """Walk policy 2 (additive complexity minimisation) on the three kernels
    against the oracle, including best_nnz, from a walked (non-minimal) start."""
    if fmt == (6, 7, 9) and mode == tfg.TFG_MODE_Z2:
        pytest.skip("one mode suffices at rank 378")
    steps0 = 1500 if fmt != (6, 7, 9) else 150
    src = oracle.Walkers(fmt, naive_start(*fmt), np.arange(1), seed=3, mode=mode, plateau_len=200).walk(steps0)
    start = src.scheme(0)
    steps = 1500 if fmt != (6, 7, 9) else 300
    # policy 2 never grows the rank: one spare slot keeps (3,3,3) within 32 slots
    W = gpu_walkers(fmt, mode, start, nw, 9, steps, chunks=2, walk_policy=2, mapping=lanes, r_slack=1)
    info, slots, best = W.read_walkers(0, nw)
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=9, mode=mode, policy=2, r_slack=1).walk(steps, THREADS)
    assert_parity(info, slots, best, ref, range(nw), f"policy 2 {fmt} G={lanes} mode={mode}")
    assert np.array_equal(info["best_nnz"], ref.info["best_nnz"].astype(np.uint32))
    assert W.verify_all() == 0
    W.close()
