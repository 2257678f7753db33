"""The tile autotuner (jagp_autotune): its choices come from the candidate
sets, and every result (log|Psi|, positions after sweeps, e_L, acceptance) is
identical with and without tuning, since the candidates change only how the
outputs are tiled, never the order of a sum."""
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
                assert t["umma_bn_left"] in (16, 32, 48, 64, 80, 96, 128)
                assert t["umma_bn_right"] in (16, 32, 48, 64, 80, 96)
                assert t["umma_stages_left"] in (0, 2, 3) and t["umma_stages_right"] in (0, 2, 3)
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
