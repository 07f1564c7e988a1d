"""The learned-closure loop on the GPU (paper_0808_4078_gb300.closure_study): a collisionless 3D
run's moments train the network, which then sets the return-current drag of a 2D run.

Parity of the two device steps the loop adds:
  * pic_closure_samples against oracle.closure.samples (FP64 on both sides; the device rounds the
    results to FP32): the same samples kept, in the same order, features and labels to FP32
    rounding;
  * pic_mlp_fit_norm against oracle.mlp.feature_norm.

The loop at crop size (3D 64 x 64 x 128 cells, 2D 64 x 64, 8 particles per cell and species,
hot beam T_perp = 0.2, 2000 steps, current filter on):
  * the 3D run's transverse magnetic energy has an exponential stage (0.05 < Gamma < 0.2);
  * the windows keep most samples and both networks learn them (R^2 > 0.5);
  * the gain: the 2D runs driven by either network (9 inputs, and 8 without W_ES) reach the 3D
    run's peak magnetic energy per unit volume far more closely than the 2D run without drag
    and than the best constant Krook rate of {0.01, 0.03, 0.1, 0.3, 1} (log-ratio error at most
    half of theirs; measured ~0.9 against >= 4.6).
The growth rate is reported, not asserted: no 2D run of this size has an exponential stage (the
network-driven runs rise within the first few 1/w_p, the others stay at the noise level).
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    import __graft_entry__ as ge
    ge.build()
    import paper_0808_4078_gb300 as pic
    return pic


def test_samples_kernel_matches_oracle(pic):
    import torch
    from oracle import closure
    from paper_0808_4078_gb300 import closure_study as cs
    rng = np.random.default_rng(9)
    nsnap, nc, window = 23, 300, 5                     # 4 windows, 3 snapshots left over
    rows = rng.normal(size=(nsnap, 12, nc)).astype(np.float32)
    rows[:, 3] = (-0.1 + 0.05 * rng.normal(size=(nsnap, nc))).astype(np.float32)
    rows[:, 3, ::7] = 1e-3                             # stopped return current: dropped
    feat, lab = cs.training_set(torch.from_numpy(rows).cuda(), window, 0.05, 0.01)
    f_o, l_o = closure.samples(rows.astype(np.float64), window, 0.05, 0.01)
    assert feat.shape[1] == l_o.size and 0 < l_o.size < 4 * nc
    f_g, l_g = feat.double().cpu().numpy(), lab.double().cpu().numpy()
    assert np.allclose(f_g, f_o, rtol=2e-7, atol=1e-7)
    assert np.allclose(l_g, l_o, rtol=1e-6, atol=1e-7)


def test_fit_norm_matches_oracle(pic):
    import torch
    from oracle import mlp
    from paper_0808_4078_gb300 import closure_study as cs
    rng = np.random.default_rng(10)
    x = (rng.normal(size=(9, 5001)) * np.linspace(0.1, 4, 9)[:, None] + np.arange(9)[:, None]).astype(np.float32)
    x[4] = 2.5                                          # constant feature: deviation 1
    for nin in (9, 8):
        mu, sd = cs.fit_norm(torch.from_numpy(x).cuda(), nin)
        mo, so = mlp.feature_norm(x[:nin].T.astype(np.float64))
        assert np.allclose(mu[:nin], mo, rtol=1e-6, atol=1e-6)
        assert np.allclose(sd[:nin], so, rtol=1e-6)
        assert np.all(mu[nin:] == 0) and np.all(sd[nin:] == 1)


def test_closure_loop_gain(pic):
    from paper_0808_4078_gb300 import closure_study as cs
    res = cs.run_study(64, 64, 128, 8, 2000, train_steps=1500)
    g3 = res["run3d"]["gamma"]
    assert 0.05 < g3 < 0.2, g3
    assert res["samples"]["n"] > 0.9 * res["samples"]["of"]
    for nin in (9, 8):
        assert res[f"train{nin}"]["r2"] > 0.5, res[f"train{nin}"]
    e0 = res["run2d_nu0"]["level_log"]
    ec = res["best_const_level"]["level_log"]
    for nin in (9, 8):
        en = res[f"run2d_net{nin}"]["level_log"]
        assert math.isfinite(en) and en < 0.5 * min(e0, ec), (nin, en, e0, ec)
