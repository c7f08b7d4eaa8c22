"""Pin of the oracle's threaded row split.

The oracle can split the rows (or row pairs, or slabs) of a sweep into
contiguous chunks, one per thread, to run faster on many host cores.  Every
factor of the Trotter product (Sec. 2) acts on disjoint pairs, and each site's
arithmetic does not depend on which thread does it, so any split must give
the single-thread result bit for bit.  A chunk bound that is off by one would
apply one row's rotations twice or not at all; that keeps the norm, so only a
bitwise comparison catches it.

Sizes are odd and large enough that every thread count below actually splits
(the oracle runs a range inline when it has fewer than two items per thread),
so chunk bounds fall inside the range and between both parities' pairs.
"""
import numpy as np
import pytest

import oracle

THREADS = (2, 3, 7, 16)
NX, NY = 37, 71           # rows: 71 >= 2 * 16; y pairs (71 - p) / 2 = 35 >= 2 * 16
NX3, NY3, NZ3 = 5, 7, 67   # z pairs (67 - p) / 2 = 33 >= 2 * 16; slabs 67; rows 469


def rand2(seed):
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((NY, NX))
    im = rng.standard_normal((NY, NX))
    V = rng.uniform(-2.0, 2.0, (NY, NX))
    return re, im, V


def rand3(seed):
    rng = np.random.default_rng(seed)
    shp = (NZ3, NY3, NX3)
    return rng.standard_normal(shp), rng.standard_normal(shp), rng.uniform(-2.0, 2.0, shp)


def same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y), "threaded result differs from one thread"


@pytest.mark.parametrize("nt", THREADS)
@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("parity", [0, 1])
def test_sweep_split_is_bitwise_single_thread(nt, axis, parity):
    re, im, _ = rand2(1)
    same(oracle.sweep(re, im, axis, parity, 0.3, nthreads=nt),
         oracle.sweep(re, im, axis, parity, 0.3, nthreads=1))


@pytest.mark.parametrize("nt", THREADS)
def test_phase_split_is_bitwise_single_thread(nt):
    re, im, V = rand2(2)
    same(oracle.phase(re, im, V, 0.05, nthreads=nt), oracle.phase(re, im, V, 0.05, nthreads=1))


@pytest.mark.parametrize("nt", THREADS)
@pytest.mark.parametrize("order", [1, 2, 4])
def test_evolve_split_is_bitwise_single_thread(nt, order):
    re, im, V = rand2(3)
    same(oracle.evolve(re, im, V, 0.05, 0.025, 3, order=order, nthreads=nt),
         oracle.evolve(re, im, V, 0.05, 0.025, 3, order=order, nthreads=1))


@pytest.mark.parametrize("nt", THREADS)
def test_driven_split_is_bitwise_single_thread(nt):
    re, im, V0 = rand2(4)
    V1 = np.random.default_rng(5).uniform(-1.0, 1.0, V0.shape)
    a = np.array([0.3, -0.7, 1.1])
    same(oracle.evolve_driven(re, im, V0, V1, a, 0.05, 0.025, nthreads=nt),
         oracle.evolve_driven(re, im, V0, V1, a, 0.05, 0.025, nthreads=1))


@pytest.mark.parametrize("nt", THREADS)
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("parity", [0, 1])
def test_sweep3_split_is_bitwise_single_thread(nt, axis, parity):
    re, im, _ = rand3(6)
    same(oracle.sweep3(re, im, axis, parity, 0.3, nthreads=nt),
         oracle.sweep3(re, im, axis, parity, 0.3, nthreads=1))


@pytest.mark.parametrize("nt", THREADS)
def test_evolve3_split_is_bitwise_single_thread(nt):
    re, im, V = rand3(7)
    same(oracle.evolve3(re, im, V, 0.05, 0.025, 2, nthreads=nt),
         oracle.evolve3(re, im, V, 0.05, 0.025, 2, nthreads=1))


@pytest.mark.parametrize("nt", THREADS)
def test_adjoint_split_is_bitwise_single_thread(nt):
    re, im, V = rand2(8)
    tr, ti, _ = rand2(9)
    g1, f1, c1 = oracle.adjoint_grad(re, im, tr, ti, V, 0.05, 0.025, 3, nthreads=1)
    gn, fn, cn = oracle.adjoint_grad(re, im, tr, ti, V, 0.05, 0.025, 3, nthreads=nt)
    assert np.array_equal(g1, gn)
    assert f1 == fn and c1 == cn


def check_all_splits():
    """Every test above at every thread count (the planted-mistake test runs
    this against a mutant oracle)."""
    for nt in THREADS:
        for axis in "xy":
            for parity in (0, 1):
                test_sweep_split_is_bitwise_single_thread(nt, axis, parity)
        test_phase_split_is_bitwise_single_thread(nt)
        for order in (1, 2, 4):
            test_evolve_split_is_bitwise_single_thread(nt, order)
        test_driven_split_is_bitwise_single_thread(nt)
        for axis in (0, 1, 2):
            for parity in (0, 1):
                test_sweep3_split_is_bitwise_single_thread(nt, axis, parity)
        test_evolve3_split_is_bitwise_single_thread(nt)
        test_adjoint_split_is_bitwise_single_thread(nt)
