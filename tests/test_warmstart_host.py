"""Host logic of the learned warm start (no GPU): the held-out split, the
step-size schedule, the data-set file round trip, the trained-range
fallback, and the H2 workload the data set is built from."""
import math

import numpy as np
import pytest

from paper_2003_01833_gb300 import warmstart as WS
from paper_2003_01833_gb300 import workloads as W


def test_split_holds_out_every_fourth_geometry():
    tr, te = WS.split(32)
    assert te == [1, 5, 9, 13, 17, 21, 25, 29]
    assert sorted(tr + te) == list(range(32)) and not set(tr) & set(te)
    R = W.h2_bond_lengths()
    # held-out bond lengths lie inside the trained range (interpolation)
    assert R[tr].min() < R[te].min() and R[te].max() < R[tr].max()


def test_cosine_schedule_endpoints():
    lr = WS.cosine_lr(3e-3, 100)
    assert lr(1) == pytest.approx(3e-3)
    assert lr(51) == pytest.approx(1.5e-3)
    assert 0 < lr(100) < 1e-5
    assert all(lr(k) >= lr(k + 1) for k in range(1, 100))


def test_data_set_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    recs = [{"R": 1.0 + i, "n": 5, "w_sum": 2.5, "psi": rng.normal(size=5).astype(np.float32), "eps": -0.4,
             "e_total": -1.1, "converged": True, "scf_steps": 5, "gi_steps": 20, "seconds": 0.3} for i in range(3)]
    p = tmp_path / "d.npz"
    WS.save(recs, str(p))
    back = WS.load(str(p))
    assert len(back) == 3
    for a, b in zip(recs, back):
        for k, v in a.items():
            if k == "psi":
                np.testing.assert_array_equal(v, b[k])
            else:
                assert v == b[k]


def test_prediction_outside_the_trained_range_falls_back():
    """Outside the bond lengths the models saw, predict() keeps the
    superposition start and touches no model or device."""
    wl = W.hydrogen_molecule(2.4, tol_m=1e-4)
    assert WS.predict(None, None, wl, R_range=(1.0, 2.0)) is None


def test_h2_workload():
    wl = W.hydrogen_molecule(1.4, tol_m=1e-4)
    w = wl.mesh.w
    assert wl.n_elec == 2.0 and wl.psi.shape[0] == 1
    assert abs(wl.e_zz - 1.0 / 1.4) < 1e-15
    assert abs(np.sum(wl.psi[0] ** 2 * w) - 1.0) < 1e-12
    assert abs(np.sum(wl.rho * w) - 2.0) < 1e-3
    np.testing.assert_allclose(wl.meta["nuclei"], [[-0.7, 0, 0], [0.7, 0, 0]])
    # the sigma_g start is symmetric under x -> -x
    x = wl.mesh.xyz
    i = np.lexsort((x[2], x[1], x[0]))
    j = np.lexsort((x[2], x[1], -x[0]))
    np.testing.assert_allclose(wl.psi[0][i], wl.psi[0][j], rtol=1e-12)


def test_mlp_init_is_glorot_and_float32():
    p = W.mlp_init(3)
    assert p.size == 1377
    np.testing.assert_array_equal(p, p.astype(np.float32).astype(np.float64))
    W1, W2, W3 = p[:256], p[288:1312], p[1344:1376]
    assert np.abs(W1).max() <= math.sqrt(6 / 40) and np.abs(W2).max() <= math.sqrt(6 / 64)
    assert np.abs(W3).max() <= math.sqrt(6 / 33)
    assert np.all(p[256:288] == 0) and np.all(p[1312:1344] == 0) and p[-1] == 0


def test_co_data_set_geometries():
    """The CO density data set: 32 seeded bond lengths in [1.9, 2.4] Bohr,
    held-out ones inside the trained range; the workload puts C and O on the
    x axis at -R/2 and R/2, and its superposition density integrates to
    N_e = 14 on the tol_m = 3e-6 mesh."""
    R = W.co_bond_lengths()
    assert len(R) == 32 and R.min() >= 1.9 and R.max() <= 2.4 and np.all(np.diff(R) > 0)
    tr, te = WS.split(32)
    assert R[tr].min() < R[te].min() and R[te].max() < R[tr].max()
    wl = W.carbon_monoxide_scf(tol_m=3e-4, R=2.2)
    np.testing.assert_allclose(wl.meta["nuclei"], [[-1.1, 0, 0], [1.1, 0, 0]])
    assert wl.meta["R"] == 2.2 and wl.n_elec == 14.0
    assert abs(np.sum(wl.rho * wl.mesh.w) - 14.0) < 1e-2


def test_split_leaves_out_runs_that_did_not_converge():
    """The CO data set keeps only converged SCF runs; every fourth of those
    (in sorted order, starting with the second) is held out."""
    from paper_2003_01833_gb300 import warmstart as WS

    conv = [True, False, True, True, True, False, True, True, True, True]
    tr, te = WS.split_converged([{"converged": c} for c in conv])
    usable = [i for i, c in enumerate(conv) if c]  # 0 2 3 4 6 7 8 9
    assert te == [usable[1], usable[5]] == [2, 7]
    assert sorted(tr + te) == usable and not set(tr) & set(te)
