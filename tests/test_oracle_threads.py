"""The oracle's threaded outer loops change no bit of its results.

With threads, a forward's rows and an adjoint's columns are cut into ranges,
one per thread; each output is still one sum in the single-threaded order.
So forward, adjoint, the power iteration and FISTA (which call them) must
give bitwise the single-threaded results, for every kind, with gains and
weights, for any thread count -- including more threads than outputs."""
import numpy as np
import pytest

import oracle
from paper_1310_2078_gb300 import synth


def _problem(d, threads):
    return oracle.Problem(d["uvw"], d["lm"], d["sigma"], d["kind"], d["weights"], d["ant_pair"],
                          d["gains"], threads=threads)


@pytest.mark.parametrize("threads", [2, 3, 8, 1000])
def test_threaded_oracle_is_bitwise_single_threaded(threads):
    d = synth.random_problem(41, 301, 157, kinds=(0, 1, 2), gains=True, weights=True)
    P1, Pt = _problem(d, 1), _problem(d, threads)
    rng = np.random.default_rng(3)
    x = np.abs(rng.normal(size=157))
    r = rng.normal(size=301) + 1j * rng.normal(size=301)
    assert np.array_equal(oracle.forward(P1, x), oracle.forward(Pt, x))
    assert np.array_equal(oracle.adjoint(P1, r), oracle.adjoint(Pt, r))
    rows, cols = np.array([300, 0, 17, 17]), np.array([156, 3])
    assert np.array_equal(oracle.forward(P1, x, rows=rows), oracle.forward(Pt, x, rows=rows))
    assert np.array_equal(oracle.adjoint(P1, r, cols=cols), oracle.adjoint(Pt, r, cols=cols))
    L1, i1 = oracle.power(P1, max_iter=15)
    Lt, it = oracle.power(Pt, max_iter=15)
    assert (L1, i1) == (Lt, it)
    V = oracle.forward(P1, x)
    lam = 0.05 * oracle.adjoint(P1, V).max()
    img1, s1 = oracle.fista(P1, V, lam, L1, 12, tol=1e-9)
    imgt, st = oracle.fista(Pt, V, lam, L1, 12, tol=1e-9)
    assert np.array_equal(img1, imgt) and s1 == st


def test_threaded_oracle_rejects_bad_indices():
    d = synth.random_problem(42, 20, 10)
    Pt = _problem(d, 4)
    with pytest.raises(ValueError):
        oracle.forward(Pt, np.ones(10), rows=np.array([0, 20]))
    with pytest.raises(ValueError):
        oracle.adjoint(Pt, np.ones(20, complex), cols=np.array([-1]))
