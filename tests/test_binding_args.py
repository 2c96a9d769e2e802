"""CPU checks of the Python binding's argument handling: bad arguments are
refused before any device work (no GPU needed)."""
import numpy as np
import pytest
import torch

from paper_2605_30267_gb300 import binding as B


def test_unknown_cost_kind_and_method_are_refused():
    X = torch.zeros(4, 3)
    with pytest.raises(ValueError):
        B.problem_points(X, X, kind="euclid")
    with pytest.raises(ValueError):
        B.solve(torch.zeros(3, 3), None, None, eps=1e-2, method="fast")
    with pytest.raises(ValueError):
        B.solve_points(X, X, None, None, eps=1e-2, method="accelerated")
    with pytest.raises(ValueError):
        B.problem_host(np.ones(4) / 4, np.ones(4) / 4, X=np.zeros((4, 3), np.float32),
                       Y=np.zeros((4, 3), np.float32), kind="l1")


def test_host_tensors_are_refused_where_device_ones_are_needed():
    with pytest.raises(TypeError, match="CUDA tensor"):
        B.problem_dense(torch.zeros(3, 3, dtype=torch.float32))
    with pytest.raises(TypeError, match="CUDA tensor"):
        B.problem_points(torch.zeros(4, 2), torch.zeros(5, 2), kind="cosine")


def test_unknown_parameter_is_refused():
    with pytest.raises(TypeError):
        B.default_params(epsilon=1e-2)
    p = B.default_params(eps=0.5, tol=1e-7, method=B.PLAIN)
    assert p.eps == 0.5 and p.tol == 1e-7 and p.method == B.PLAIN


def test_host_problem_struct():
    a = np.full(3, 1 / 3)
    b = np.full(5, 1 / 5)
    X = np.random.default_rng(0).random((3, 2)).astype(np.float32)
    Y = np.random.default_rng(1).random((5, 2)).astype(np.float32)
    pr = B.problem_host(a, b, X=X, Y=Y, kind="cosine", scale_to_max=True)
    assert (pr.n, pr.m, pr.d) == (3, 5, 2)
    assert pr.cost_kind == B.COST_COSINE and pr.cost_scale == B.SCALE_MAX_TO_ONE
    C = np.random.default_rng(2).random((3, 5)).astype(np.float32)
    pd = B.problem_host(a, b, C=C)
    assert pd.cost_kind == B.COST_DENSE and pd.ldc == 5


def test_device_vectors_are_checked_before_the_library_sees_them():
    B._check_vec(None, 5, "f_out")                       # left to the library's null check
    with pytest.raises(TypeError, match="CUDA float64"):
        B._check_vec(torch.zeros(5, dtype=torch.float64), 5, "f_out")
    with pytest.raises(TypeError, match="CUDA float64"):
        B._check_vec(np.zeros(5), 5, "g_out")


def test_noalloc_wrapper_checks_its_vectors():
    # refused before the library is called: host, wrong dtype
    pr = B.accsink_problem()
    pr.n, pr.m = 4, 6
    with pytest.raises(TypeError, match="CUDA float64"):
        B.accsink_col_lse_noalloc(pr, 1e-2, torch.zeros(4, dtype=torch.float64),
                                  torch.zeros(6, dtype=torch.float64))
    with pytest.raises(TypeError, match="CUDA float64"):
        B.accsink_col_lse_noalloc(pr, 1e-2, np.zeros(4), np.zeros(6))
