"""Host logic of the branch-and-bound driver and of the warm-start parameter
block (no GPU): branching choice, incumbent support, parameter layout."""
import numpy as np
import pytest

from oracle import mlp


def test_branch_variable_is_the_largest_free_coordinate():
    from paper_2603_01306_gb300.bnb import _branch_var
    beta = np.array([0.5, -3.0, 2.0, 0.0, -2.5])
    fix = np.array([0, -1, 1, 0, 0], dtype=np.int8)    # |beta_1| is largest but in J0; beta_2 is in J1
    assert _branch_var(beta, fix) == 4
    assert _branch_var(np.array([0.0, 1.0]), np.array([0, 1], dtype=np.int8)) == -1   # nothing free and nonzero


def test_incumbent_support_keeps_j1_and_fills_by_magnitude():
    from paper_2603_01306_gb300.bnb import _incumbent_fix
    beta = np.array([0.1, -0.9, 0.05, 0.7, 0.0, -0.3])
    fix = np.array([1, 0, 0, 0, 0, -1], dtype=np.int8)
    f = _incumbent_fix(beta, fix, k=3)
    assert list(np.flatnonzero(f == 1)) == [0, 1, 3]   # J1 first, then |beta| descending
    assert np.all(f[[2, 4, 5]] == -1)                  # everything else fixed to zero
    # fewer free nonzeros than k: the support stays smaller, zeros are never added
    f2 = _incumbent_fix(np.array([0.0, 0.2, 0.0]), np.zeros(3, dtype=np.int8), k=3)
    assert list(np.flatnonzero(f2 == 1)) == [1]


def test_parameter_block_layout_and_initial_network():
    from paper_2603_01306_gb300.binding import MLP_NPARAM, MLP_NTRAIN
    from paper_2603_01306_gb300.warmstart import init_params
    assert (MLP_NTRAIN, MLP_NPARAM) == (mlp.N_TRAIN, mlp.N_PARAM)
    th = init_params(seed=3)
    assert th.shape == (MLP_NPARAM,)
    W1, b1, W2, b2, w3, b3, shift, scale = mlp.unpack(th)
    assert np.all(w3 == 0) and b3 == 0                 # the untrained network is the parent start
    assert np.all(shift == 0) and np.all(scale == 1)
    assert W1.std() == pytest.approx(np.sqrt(2 / 5), rel=0.2)
    assert W2.std() == pytest.approx(np.sqrt(2 / 64), rel=0.1)
    F = np.random.default_rng(0).standard_normal((9, 5))
    out, _ = mlp.forward(th, F)
    assert np.all(out == 0)
