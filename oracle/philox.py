"""Philox4x32-10 counter-based generator and the uniform used by every event.

Oracle (test infrastructure only).  Written from the published definition of
Philox (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): a 4x32-bit counter, a 2x32-bit key, ten rounds of two
32x32->64 multiplications with the multipliers 0xD2511F53 and 0xCD9E8D57,
the key bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.

Draw rule of the simulator: the uniform of event `e` of trajectory `t` under
64-bit `seed` uses key (seed_lo, seed_hi), counter (t_lo, t_hi, e, 0); with
the first two output words w0, w1,
    u = ((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53     (53 random bits, in [0,1)).

Parity: the block function is pinned to the published known-answer vectors
of Philox4x32-10 (Random123's known-answer tests; tests/golden/
philox4x32_10_kat.txt), and the derived uniforms by statistical tests
(moments, Kolmogorov-Smirnov, independence of neighbouring counters) in
tests/test_oracle_rng.py.  The device generator is compared with this one
bit for bit.
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """One block: ctr = 4 uint32, key = 2 uint32 (python ints)."""
    c0, c1, c2, c3 = [x & MASK for x in ctr]
    k0, k1 = key[0] & MASK, key[1] & MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def uniform(seed: int, traj: int, event: int) -> float:
    w = philox4x32_10((traj & MASK, (traj >> 32) & MASK, event & MASK, 0),
                      (seed & MASK, (seed >> 32) & MASK))
    return ((w[0] >> 5) * 67108864 + (w[1] >> 6)) * (1.0 / 9007199254740992.0)


def philox4x32_10_np(c0, c1, c2, c3, k0, k1):
    """Vectorised block over numpy uint64 arrays holding 32-bit values."""
    c0, c1, c2, c3 = [np.asarray(x, dtype=np.uint64) & MASK for x in (c0, c1, c2, c3)]
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    m0, m1 = np.uint64(M0), np.uint64(M1)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def uniforms(seed: int, traj, events):
    """u[traj_i, event_j] for arrays of trajectory indices and event ids."""
    t = np.asarray(traj, dtype=np.uint64)[:, None]
    e = np.asarray(events, dtype=np.uint64)[None, :]
    t, e = np.broadcast_arrays(t, e)
    w0, w1, _, _ = philox4x32_10_np(t & np.uint64(MASK), t >> np.uint64(32), e,
                                     np.zeros_like(t), seed & MASK, (seed >> 32) & MASK)
    hi = (w0 >> np.uint64(5)).astype(np.float64)
    lo = (w1 >> np.uint64(6)).astype(np.float64)
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0)
