"""The learned surrogate: trained on batched-solver runs by the library's MLP kernels, it
predicts held-out runs' diffraction and spin-flip populations (log10) far better than the
trained-set mean, answers orders of magnitude faster than the solver, and hands
out-of-range parameters to the solver."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SMALL = dict(grid=(128, 64), nsteps=400, env_scale=0.2)


@pytest.fixture(scope="module")
def trained():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2307_01571_gb300 import _build
    _build.build()
    from paper_2307_01571_gb300 import surrogate as S
    X = S.draw_params(640, seed=1)
    Y, secs = S.solve(X, batch=320, **SMALL)
    n_tr = 576
    sur = S.Surrogate(seed=0)
    sur.fit(X[:n_tr], Y[:n_tr], steps=2500, batch=128, lr=2e-3)
    return S, sur, X, Y, n_tr, secs


def test_heldout_error_beats_constant_predictor(trained):
    S, sur, X, Y, n_tr, _ = trained
    pred = sur.predict(X[n_tr:])
    err = S.heldout_error(pred, Y[n_tr:])
    base = S.heldout_error(np.tile(Y[:n_tr].mean(0), (len(X) - n_tr, 1)), Y[n_tr:])
    for k in ("log10_P_bragg", "log10_P_bragg_same_spin", "log10_P_bragg_flip"):
        assert err[k]["rms"] < 0.25 * base[k]["rms"], (k, err[k], base[k])
    assert np.all(np.isfinite(pred))


def test_surrogate_is_much_faster_than_the_solver(trained):
    S, sur, X, Y, n_tr, secs = trained
    Xh = X[n_tr:]
    sur.predict(Xh)
    t0 = time.perf_counter()
    for _ in range(10):
        sur.predict(Xh)
    t_pred = (time.perf_counter() - t0) / (10 * len(Xh))
    t_solve = secs / len(X)
    assert t_solve / t_pred > 100, (t_solve, t_pred)


def test_out_of_domain_rows_fall_back_to_the_solver(trained):
    S, sur, X, Y, n_tr, _ = trained
    rows = np.array([X[n_tr], [30.0, X[n_tr, 1], X[n_tr, 2], X[n_tr, 3], X[n_tr, 4]]])
    out, used = sur.predict_or_solve(rows, **SMALL)
    assert list(used) == [False, True]
    direct, _ = S.solve(rows[1:], **SMALL)
    assert np.array_equal(out[1], direct[0])
