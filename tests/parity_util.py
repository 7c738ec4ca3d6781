"""Shared helpers for the GPU-vs-oracle parity tests (inputs and comparisons only)."""
import numpy as np

# one iteration from identical state: norm-wise relative error per vector
ONE_STEP_RTOL = 1e-5
# final exploitability after T iterations (see test_gpu_parity for the reading)
EXPL_RTOL = 1e-3


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = max(np.linalg.norm(b), 1e-300)
    return float(np.linalg.norm(a - b) / den)


def random_state(o, p, rng, scale=1.0, t=5):
    """Seeded state for player p of an oracle game: regrets, a behavioural
    strategy on each infoset's simplex, positive average sums."""
    S = o.S[p]
    r = rng.standard_normal(S) * scale
    r[rng.uniform(size=S) < 0.2] = 0.0
    ps, na = o.infosets(p)
    b = np.zeros(S)
    off = 0
    for n in na:
        w = rng.uniform(0.05, 1.0, n)
        b[off:off + n] = w / w.sum()
        off += n
    xbar = np.abs(rng.standard_normal(S + 1)) * 3.0
    return r, b, xbar, t


def strategy_mismatch_ok(b_gpu, b_orc, r_orc_next, na, tol=1e-5, tie=1e-6):
    """Compare next strategies infoset by infoset.  Where the oracle's
    positive-regret sum is at the level of rounding noise, regret matching's
    zero test may legitimately go either way (uniform vs. a vertex), so only
    validity is checked there.  Returns the number of mismatching infosets."""
    off = 0
    scale = max(1.0, np.abs(r_orc_next).max())
    bad = 0
    for n in na:
        sl = slice(off, off + n)
        pos = np.maximum(r_orc_next[sl], 0).sum()
        if pos > tie * scale:
            bad += int(np.abs(b_gpu[sl] - b_orc[sl]).max() > tol)
        else:
            assert abs(b_gpu[sl].sum() - 1.0) < 1e-5 and (b_gpu[sl] >= 0).all()
        off += n
    return bad
