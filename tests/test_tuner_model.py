"""CPU checks of the committed learned-tuner model and its training data.

The network is evaluated with the FP64 oracle's forward pass (independent of
the GPU kernels that trained it): it must rank the configurations of its own
training rows (GB300 full-search timings of the density sweep) close to the
measured best over all timed configurations, of which it ranks the candidates
(those within 10 % of some row's best)."""
import numpy as np
import pytest

import oracle
from paper_2512_03565_gb300 import tuner


def test_oracle_targets_are_relative_log_times():
    """Hand-built rows: the best entry is 0, the others log of their ratio to
    it; untimed (NaN), zero and negative entries are masked; a row with no
    valid entry is all masked; scaling a row leaves its targets unchanged."""
    oracle.build()
    T = np.array([[2.0, 1.0, np.nan, 4.0], [3.0, 3.0, 6.0, 1.5], [np.nan, 0.0, -1.0, np.inf]])
    Y, M = oracle.tuner_targets(T)
    np.testing.assert_allclose(Y[0], [np.log(2.0), 0.0, 0.0, np.log(4.0)], rtol=1e-15)
    np.testing.assert_allclose(Y[1], [np.log(2.0), np.log(2.0), np.log(4.0), 0.0], rtol=1e-15)
    np.testing.assert_array_equal(M, [[1, 1, 0, 1], [1, 1, 1, 1], [0, 0, 0, 0]])
    np.testing.assert_array_equal(Y[2], 0.0)
    Y2, M2 = oracle.tuner_targets(T * 7.25)
    np.testing.assert_allclose(Y2[:2], Y[:2], atol=1e-15)
    np.testing.assert_array_equal(M2, M)


def test_oracle_standardization_is_numpy_mean_and_std():
    """Against numpy's mean and population std (a textbook routine); a
    constant column keeps std 1 and standardises to 0."""
    oracle.build()
    rng = np.random.default_rng(4)
    X = rng.normal(3.0, 2.0, size=(200, 16))
    X[:, 5] = 4.0
    Xs, mean, sd = oracle.standardize(X)
    np.testing.assert_allclose(mean, X.mean(axis=0), rtol=1e-13)
    want = X.std(axis=0)
    want[5] = 1.0
    np.testing.assert_allclose(sd, want, rtol=1e-12)
    np.testing.assert_allclose(Xs, (X - mean) / sd, rtol=1e-13, atol=1e-14)
    np.testing.assert_array_equal(Xs[:, 5], 0.0)


def test_candidates_are_the_configurations_near_some_best():
    # config 0 best in row 0; config 1 within 25 % (not 10 %) in row 1; config 2 never within 25 %;
    # config 3 best in row 1 but missing (NaN) in row 0
    T = np.array([[1.0, 1.5, 2.0, np.nan], [2.0, 1.2, 3.0, 1.0]])
    np.testing.assert_array_equal(tuner.candidates(T, near=1.25), [True, True, False, True])
    np.testing.assert_array_equal(tuner.candidates(T, near=1.1), [True, False, False, True])


def test_committed_model_ranks_its_training_rows():
    import os
    path = os.path.join(os.path.dirname(tuner.MODEL_PATH), "tuner_data.npz")
    z = np.load(path)
    X, T, names = z["X"], z["T"], [str(v) for v in z["names"]]
    z2 = np.load(tuner.MODEL_PATH)
    params, mean, std, C = z2["params"].astype(np.float64), z2["mean"], z2["std"], int(z2["C"])
    out_names = [str(v) for v in z2["names"]]
    # the outputs are the candidate configurations of the training timings, in order
    keep = tuner.candidates(T)
    assert out_names == [n for n, k in zip(names, keep) if k]
    assert params.shape[0] == oracle.mlp_nparams(C) and C == len(out_names)
    cols = np.array([names.index(n) for n in out_names])
    oracle.build()
    Y = oracle.mlp_forward(params, C, (X - mean) / std)
    M = tuner.valid(T)
    regrets = []
    for r in range(X.shape[0]):
        p = np.where(M[r, cols] > 0, Y[r], np.inf)
        k = int(cols[int(np.argmin(p))])
        regrets.append(T[r, k] / np.nanmin(np.where(M[r] > 0, T[r], np.nan)))
    regrets = np.array(regrets)
    assert np.median(regrets) <= 1.02
    assert np.mean(regrets) <= 1.05
