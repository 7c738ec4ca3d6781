"""The bounded-wait failure path, on the GPU, without faulting or hanging it.

Every wait of a unit of work for the units it depends on is bounded on the
device; when the bound runs out the kernel records the timeout in the
context's error word and returns, and the host reports CFR_ERR_TIMEOUT.  Here
the bound is made tiny through the `wait_us` load option (1 us), so that the
large game's internal units, which wait for dozens of leaf units, give up.
Nothing is left waiting: the kernels return, the context refuses further
work, and a new context on the same device runs normally.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ERR_TIMEOUT, ERR_STATE = -4, -5


@pytest.fixture(scope="module")
def cfr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2605_14277_b300 import cfr as C
    return C


def test_wait_that_runs_out_reports_timeout_and_poisons_the_context(cfr):
    from paper_2605_14277_b300 import games as G
    tree = G.large_random_game(3)
    s = cfr.Solver(tree, wait_us=1)
    s.iterate(20, "dcfr")
    with pytest.raises(cfr.CFRError) as e:
        s.sync()
    assert e.value.status == ERR_TIMEOUT
    for call in (lambda: s.iterate(1, "dcfr"), s.sync, s.exploitability, lambda: s.get_state(1)):
        with pytest.raises(cfr.CFRError) as e:
            call()
        assert e.value.status == ERR_STATE
    s.close()
    # a fresh context on the same device (default bound) works and is exact
    a = cfr.Solver(G.poker_game())
    b = cfr.Solver(G.poker_game())
    a.iterate(70, "cfr+")
    b.iterate(70, "cfr+")
    for p in (1, 2):
        assert np.array_equal(a.get_state(p)["r"], b.get_state(p)["r"])
    assert a.exploitability()[0] > 0


def test_kernel_launch_count(cfr):
    """One eager iteration is a parameter-table launch and L = 4 pass launches
    (per player: the staged bottom-up pass and the top-down pass).  130
    iterations = two replays of a 64-iteration graph (one table launch and
    64 L passes each) and two eager iterations (one table launch for both)."""
    from paper_2605_14277_b300 import games as G
    one = cfr.Solver(G.poker_game(), passes=2)
    one.iterate(1, "dcfr")
    L = one.kernel_launches() - 1
    assert L == 4
    s = cfr.Solver(G.poker_game(), passes=2)
    assert s.kernel_launches() == 0
    s.iterate(130, "dcfr")
    s.sync()
    assert s.kernel_launches() == 2 * (1 + 64 * L) + (1 + 2 * L)
