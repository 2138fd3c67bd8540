"""The error model the GPU Schur-stencil parity tests use (entries stored as fp16 scaled by their
row's largest magnitude): emulated here with numpy's float16 on the oracle's B D^-1 B^T, the
stored operator's error stays inside schur_fp16_bound, and the bound is not vacuous."""
import numpy as np

import synthetic as syn
from problems import oseen, schur_fp16_bound, schur_reference


def test_fp16_row_scaled_storage_stays_within_the_bound():
    n = 4
    P = oseen(n)
    S, Sabs = schur_reference(P["A"], P["dmu"].n_dofs)
    Sd = S.toarray()
    scale = np.abs(Sd).max(axis=1)
    scale[scale == 0] = 1.0
    stored = (Sd / scale[:, None]).astype(np.float16).astype(np.float64) * scale[:, None]
    for seed in range(3):
        p = syn.uniform_pm1(20 + seed, S.shape[0])
        err = np.abs(stored @ p - S @ p)
        bound = schur_fp16_bound(S, p, n)
        assert np.all(err <= bound * (1 + 1e-12) + 1e-300)
        assert (err / bound).max() > 0.01  # in some row the storage error reaches a percent of the bound
    # and a wrong operator (one entry per row moved to the wrong neighbour) breaks it
    wrong = np.roll(Sd, 1, axis=1)
    p = syn.uniform_pm1(30, S.shape[0])
    assert np.any(np.abs(wrong @ p - S @ p) > schur_fp16_bound(S, p, n) + 5e-5 * (Sabs @ np.abs(p)))
