"""The search driver end to end on small populations: its report agrees with
the walkers' statistics, every best scheme it writes reads back and satisfies
Eq. (1) (checked by the oracle)."""
import json

import numpy as np
import pytest

import oracle
from paper_2511_20317_gb300 import search, tfg
from paper_2511_20317_gb300.workloads import naive_start, read_scheme

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2511_20317_gb300 import _build
    _build.build()
    tfg.lib()
    torch.cuda.set_device(0)


def test_search_reports_and_files(tmp_path):
    pops = [((2, 2, 2), tfg.TFG_MODE_ZT, naive_start(2, 2, 2), 512),
            ((3, 3, 3), tfg.TFG_MODE_Z2, naive_start(3, 3, 3), 256)]
    out = search.run(pops, steps=20000, chunk=7000, seed=3, plateau=2000, out_dir=str(tmp_path), quiet=True)
    assert len(out) == 2
    for (res, scheme), (fmt, mode, _, nw) in zip(out, pops):
        json.dumps(res)
        hist = res["rank_histogram"]
        assert sum(hist.values()) == nw
        assert res["lowest_rank"] == min(hist) and res["walkers_at_lowest"] == hist[res["lowest_rank"]]
        assert res["best_scheme_verified_host"] and res["device_check_failures"] == 0
        f2, s2 = read_scheme(res["file"])
        assert f2 == fmt and np.array_equal(s2, scheme) and s2.shape[0] == res["lowest_rank"]
        assert oracle.brent_valid(fmt, s2, mode)
        if mode == tfg.TFG_MODE_ZT:
            assert res["additive_complexity"] == oracle.additive_complexity(fmt, s2)
        from oracle import invariants as inv
        _, typ, _, sums = inv.isotropy_invariants(fmt, s2, mode)
        assert res["isotropy_invariants"]["type_polynomial"] == {f"{a} {b} {c}": v for (a, b, c), v in
                                                                  sorted(typ.items(), reverse=True)}
        assert res["isotropy_invariants"]["rank_sums"] == list(sums)
        if mode == tfg.TFG_MODE_Z2:
            lift = res["ternary_lifting"]
            assert lift["rank"] == res["lowest_rank"] and 1 <= lift["tried"] <= 256 and 0 <= lift["lifted"] <= lift["tried"]


def test_exploratory_search_moves_schemes_between_formats():
    """Exploratory search over (2,2,2) seeded with Strassen's scheme and formats
    reachable by Resize moves: better schemes are transferred into the other
    populations (re-seeding), every transfer beats the target's best at the
    time, and every final best scheme satisfies Eq. (1)."""
    from paper_2511_20317_gb300.workloads import strassen_start
    formats = [(2, 2, 2), (2, 2, 3), (2, 2, 4), (4, 4, 4), (2, 4, 4)]
    res, transfers = search.explore(formats, walkers=256, cycles=6, steps_per_cycle=500, seed=1,
                                    starts={(2, 2, 2): strassen_start()}, p_resize=0.9, quiet=True)
    assert transfers, "no scheme was transferred"
    naive = {f: f[0] * f[1] * f[2] for f in formats}
    last = dict(naive)
    for t in transfers:
        to = tuple(t["to"])
        assert t["rank"] < last[to]
        last[to] = t["rank"]
    for r in res:
        f = tuple(r["format"])
        assert r["best_scheme_verified_host"] and r["device_check_failures"] == 0
        assert r["lowest_rank"] <= last[f]
    by = {tuple(r["format"]): r["lowest_rank"] for r in res}
    assert by[(2, 2, 2)] == 7
    assert min(by[f] for f in formats if f != (2, 2, 2)) < min(naive[f] for f in formats if f != (2, 2, 2))


def test_exploration_with_device_resize_moves():
    """Exploration whose Resize moves run on the device, per walker (swaps,
    merges with other populations' bests, projections, products, doublings,
    extensions of blocks of walkers' best schemes): transfers happen, the
    walks go on, and every walker's best scheme satisfies Eq. (1) at the end."""
    from paper_2511_20317_gb300.workloads import strassen_start
    formats = [(2, 2, 2), (2, 2, 3), (2, 3, 2), (3, 2, 2), (2, 2, 4), (2, 4, 2), (4, 2, 2), (4, 4, 4), (2, 4, 4)]
    res, transfers = search.explore(formats, walkers=256, cycles=5, steps_per_cycle=400, seed=2,
                                    starts={(2, 2, 2): strassen_start()}, p_resize=0.9, moves_per_cycle=0,
                                    device_moves=12, r_slack=12, quiet=True)
    dev = [t for t in transfers if t.get("device")]
    assert len(dev) >= 5
    assert any(t["skipped"] < t["walkers"] for t in dev)
    assert {t["op"][:4] for t in dev} & {"swap", "merg", "doub", "exte", "prod", "proj"}
    for r in res:
        assert r["best_scheme_verified_host"] and r["device_check_failures"] == 0


def test_exploration_lifts_z2_schemes_into_ternary_populations():
    """Z_2 populations walk beside the Z_T ones; a Z_2 best below the Z_T best of its
    format is lifted to Z_T signs and re-seeds the Z_T walkers, whose final best
    is then at most the lifted rank and satisfies Eq. (1) over the integers."""
    formats = [(2, 2, 2), (3, 3, 3)]
    res, transfers = search.explore(formats, walkers=4096, cycles=4, steps_per_cycle=25000, seed=3,
                                    moves_per_cycle=0, lift_z2=True, quiet=True)
    lifts = [t for t in transfers if t["op"] == "lift"]
    assert any(tuple(t["to"]) == (3, 3, 3) for t in lifts)
    by = {(tuple(r["format"]), r["mode"]): r for r in res}
    low = min(t["rank"] for t in lifts if tuple(t["to"]) == (3, 3, 3))
    assert by[((3, 3, 3), "Z_T")]["lowest_rank"] <= low < 27
    # the Z_2 population is reported too: its lowest rank is at most the rank it lifted
    z2 = by[((3, 3, 3), "Z_2")]
    assert z2["lowest_rank"] <= low and z2["lift"]["rank"] == z2["lowest_rank"]
    assert 1 <= z2["lift"]["tried"] and 0 <= z2["lift"]["lifted"] <= z2["lift"]["tried"]
    for r in res:
        assert r["best_scheme_verified_host"] and r["device_check_failures"] == 0
