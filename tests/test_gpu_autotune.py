"""The tile autotuner (jagp_autotune) and pinned tunings (jagp_set_tuning):
the choices come from the candidate sets, and every result (log|Psi|,
positions after sweeps, e_L, acceptance) is identical with and without tuning.
The candidates change how the outputs are tiled; the chunk-major tensor-core
candidate also changes the order in which the integer slice products are
summed, which is exact while the sums stay below 2^24 (as at these sizes)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


SYSTEMS = {
    "C2": synth.config2,
    # N_up > 32: the blocked tiles are candidates of both products
    "mid-n40": lambda: synth.small_random(n_atoms=20, n_up=40, n_dn=37, per_atom=6, seed=33, side=7.0, Z=2.0),
}


@pytest.mark.parametrize("mode", ["fp64", "fp64tc", "mixed"])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_autotune_changes_no_result(torch_cuda, name, mode):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    mixed = mode == "mixed"
    prec = pg.JAGP_PREC_MIXED if mixed else pg.JAGP_PREC_FP64
    W = 96
    x0 = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=4), 5, 0.2)
    runs = []
    for tune in (False, True):
        g = pg.JAGP(sysm, W, precision=prec, seed=3, fp64_tc=mode == "fp64tc")
        r = g.positions(x0)
        if tune:
            t = g.autotune()
            assert t["tile_proposals"] in (0, 32, 64) and t["tile_refresh"] in (0, 16, 32, 64)
            if mixed:
                assert t["umma_bn_left"] in (16, 32, 48, 64)
                assert t["umma_bn_right"] in (16, 32, 48, 64)
                assert t["umma_stages_left"] in (-3, -2, -1, 0, 2, 3)
                assert t["umma_stages_right"] in (-3, -2, -1, 0, 2, 3)
                assert all(m > 0 for m in t["ms"])
            elif mode == "fp64tc":
                assert t["umma_bn_left"] in (16, 32, 48, 64) and t["umma_bn_right"] in (16, 32, 48, 64)
                assert all(m > 0 for m in t["ms"])
            else:
                assert t["umma_bn_left"] == t["umma_bn_right"] == 0
                assert t["ms"][0] > 0 and t["ms"][1] > 0
        la, _ = g.eval(r)
        eL, acc = g.sweep(r, 3, acc=True)
        info = g.info()
        runs.append([la.cpu().numpy(), r.cpu().numpy(), eL.cpu().numpy(), acc.cpu().numpy()[:, :3],
                     info["logabs"].cpu().numpy(), info["naccept"].cpu().numpy()])
        g.close()
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def test_autotune_rejects_bad_arguments(torch_cuda):
    import paper_2002_07401_gb300 as pg
    sysm = synth.config1()
    g = pg.JAGP(sysm, 8)
    with pytest.raises(pg.JagpError):
        pg.jagp_autotune(g.h, g.state, 9)   # more walkers than the handle was made for
    with pytest.raises(pg.JagpError):
        pg.jagp_autotune(g.h, g.state, 0)
    g.close()


def _run(sysm, W, prec, tuning, fp64_tc=False):
    import paper_2002_07401_gb300 as pg
    x0 = synth.jitter_walkers(synth.init_walkers(sysm, W, seed=4), 5, 0.2)
    g = pg.JAGP(sysm, W, precision=prec, seed=3, fp64_tc=fp64_tc)
    if tuning is not None:
        g.set_tuning(tuning)
    r = g.positions(x0)
    la, _ = g.eval(r)
    eL, acc = g.sweep(r, 2, acc=True)
    info = g.info()
    assert g.status() & (pg.WS_NONFINITE | pg.WS_SINGULAR) == 0
    out = [la.cpu().numpy(), r.cpu().numpy(), eL.cpu().numpy(), acc.cpu().numpy()[:, :3],
           info["logabs"].cpu().numpy(), info["naccept"].cpu().numpy()]
    g.close()
    return out


PINNED_MIXED = [
    {"tile_proposals": 0, "tile_refresh": 32, "umma_bn_left": 16, "umma_bn_right": 16,
     "umma_stages_left": 2, "umma_stages_right": 3},
    {"tile_proposals": 64, "tile_refresh": 0, "umma_bn_left": 16, "umma_bn_right": 16,
     "umma_stages_left": -1, "umma_stages_right": 3},
    {"tile_proposals": 32, "tile_refresh": 64, "umma_bn_left": 64, "umma_bn_right": 48,
     "umma_stages_left": 0, "umma_stages_right": 2},
    # chunk-major with K chunks of 32 and 16 (64- and 32-byte swizzled tiles)
    {"tile_proposals": 0, "tile_refresh": 0, "umma_bn_left": 64, "umma_bn_right": 48,
     "umma_stages_left": -2, "umma_stages_right": -3},
]


@pytest.mark.parametrize("k", range(len(PINNED_MIXED)))
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_pinned_tuning_mixed_changes_no_result(torch_cuda, name, k):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS[name]()
    base = _run(sysm, 64, pg.JAGP_PREC_MIXED, None)
    pinned = _run(sysm, 64, pg.JAGP_PREC_MIXED, PINNED_MIXED[k])
    for a, b in zip(base, pinned):
        assert np.array_equal(a, b)


def test_pinned_tuning_fp64tc_changes_no_result(torch_cuda):
    import paper_2002_07401_gb300 as pg
    sysm = SYSTEMS["mid-n40"]()
    t = {"tile_proposals": 32, "tile_refresh": 32, "umma_bn_left": 16, "umma_bn_right": 48,
         "umma_stages_left": 2, "umma_stages_right": 0}
    base = _run(sysm, 48, pg.JAGP_PREC_FP64, None, fp64_tc=True)
    pinned = _run(sysm, 48, pg.JAGP_PREC_FP64, t, fp64_tc=True)
    for a, b in zip(base, pinned):
        assert np.array_equal(a, b)


def test_set_tuning_rejects_bad_values(torch_cuda):
    import paper_2002_07401_gb300 as pg
    mixed = pg.JAGP(synth.config2(), 8, precision=pg.JAGP_PREC_MIXED)
    fp64 = pg.JAGP(synth.config2(), 8)
    fp64tc = pg.JAGP(synth.config2(), 8, fp64_tc=True)
    bad_mixed = [{"tile_proposals": 16}, {"tile_refresh": 48}, {"umma_bn_left": 24}, {"umma_bn_left": 144},
                 {"umma_bn_right": 72}, {"umma_stages_left": 1}, {"umma_stages_right": 7},
                 # six accumulators of more than 64 columns
                 {"umma_bn_left": 80}, {"umma_bn_right": 96},
                 # two chunk-major stages of six slices with K chunks of 64 fit only at 16 columns
                 {"umma_bn_right": 32, "umma_stages_right": -1}, {"umma_bn_left": 64, "umma_stages_left": -1},
                 {"umma_stages_left": -4}]
    for t in bad_mixed:
        with pytest.raises(pg.JagpError):
            mixed.set_tuning(t)
    with pytest.raises(pg.JagpError):
        fp64.set_tuning({"umma_bn_left": 32})           # no tensor-core products in plain FP64
    with pytest.raises(pg.JagpError):
        fp64tc.set_tuning({"umma_stages_left": -1})      # seven or eight slices never fit twice
    fp64.set_tuning({"tile_proposals": 64, "tile_refresh": 0})
    fp64tc.set_tuning({"umma_bn_left": 64, "umma_stages_left": 6})
    for g in (mixed, fp64, fp64tc):
        g.close()
