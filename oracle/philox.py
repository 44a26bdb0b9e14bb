"""Philox4x32-10 counter-based generator, from its published definition:
J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11.  Plain Python integers, 32-bit words.

A round maps counter (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
with multipliers M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is
bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.

Use in the quantum-jump method (the paper draws from one MersenneTwister;
a per-trajectory counter stream is used instead so that trajectories are
independent of their processing order):
    key     = (seed & 0xffffffff, seed >> 32)
    counter = (draw_index, trajectory_id, 0, 0)
    u       = (x + 0.5) * 2^-52,  x = (w1 << 20) | (w0 >> 12)   (52 bits)
so u lies strictly inside (0, 1) and the conversion is exact in FP64.
Pinned by the Random123 known-answer vectors (tests/golden/philox4x32_10_kat.txt).
"""
MASK = 0xFFFFFFFF
M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85


def philox4x32(counter, key, rounds=10):
    c0, c1, c2, c3 = (int(x) & MASK for x in counter)
    k0, k1 = (int(x) & MASK for x in key)
    for r in range(rounds):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0, p1 & MASK, (p0 >> 32) ^ c3 ^ k1, p0 & MASK)
    return c0, c1, c2, c3


def uniform(seed, traj_id, draw_index):
    """The draw_index-th uniform of trajectory traj_id, in (0, 1)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    w = philox4x32((draw_index, traj_id, 0, 0), (seed & MASK, seed >> 32))
    x = (w[1] << 20) | (w[0] >> 12)
    return (x + 0.5) * 2.0 ** -52
