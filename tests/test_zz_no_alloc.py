"""The exploitability entry point that allocates nothing.

Some callers cannot allocate device memory when they ask for a result: their
device memory belongs to another allocator (a framework's caching allocator,
an embedded runtime with a fixed budget), or an allocation's device-wide
synchronisation would stall their loop.  cfr_exploitability_batch_noalloc
serves them: it keeps its per-game scratch in a fixed device array of the
library and writes into a buffer the caller already owns.  This file is
collected last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_exploitability_matches_batch_entry_point():
    import torch
    assert torch.cuda.is_available()
    from paper_2605_14277_b300 import cfr as C
    from paper_2605_14277_b300 import games as G

    trees = [G.sized_random_game(3000 + k, 10 ** (2 + k % 3)) for k in range(6)] + [G.poker_game()]
    s = C.Solver(trees)
    s.iterate(30, "cfr+")
    # the caller's own device buffer, allocated before the call
    out = torch.full((len(trees),), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for call in range(2):
        ref, _, _ = s.exploitability_batch()
        s.exploitability_into(out.data_ptr())
        s.sync()
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-12), (call, got, ref)
        s.iterate(7, "cfr+")   # the second call sees a different state


def test_noalloc_exploitability_on_a_masked_context():
    """A context whose games are partly masked off: the best response runs
    every game, and the caller's mask is back in force afterwards."""
    import torch
    from paper_2605_14277_b300 import cfr as C
    from paper_2605_14277_b300 import games as G

    trees = [G.sized_random_game(3100 + k, 10 ** (2 + k % 3)) for k in range(5)]
    mask = [1, 0, 1, 0, 1]
    s = C.Solver(trees)
    s.iterate(12, "dcfr")
    s.iterate(9, "dcfr", active=mask)
    out = torch.full((len(trees),), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for call in range(2):
        ref, _, _ = s.exploitability_batch()
        s.exploitability_into(out.data_ptr())
        s.sync()
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-12), (call, got, ref)
        # the same mask again: no new upload, so the restored device copy counts
        s.iterate(5, "dcfr", active=mask)
    assert [s.sizes(g)["t"] for g in range(5)] == [31, 12, 31, 12, 31]


def test_noalloc_rejects_bad_arguments():
    from paper_2605_14277_b300 import cfr as C
    from paper_2605_14277_b300 import games as G

    s = C.Solver(G.rps())
    with pytest.raises(C.CFRError) as e:
        s.exploitability_into(0)
    assert e.value.status == -6
