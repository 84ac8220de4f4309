"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
Random Numbers: As Easy as 1, 2, 3", SC'11), written from its published
definition.  The quantum-trajectory method needs one uniform number per
trajectory and time step to decide jump-or-evolve and pick the channel
(Sec. 4.1, jump probabilities W(alpha -> alpha^k) dt); drawing it from a
counter-based stream makes every (trajectory, step) draw independent of how the
work is scheduled.

Counter words: (trajectory id, step low 32 bits, purpose, step high 32 bits);
key words: (seed low 32 bits, seed high 32 bits).  Purpose 0 is the jump draw.
A uniform double in [0, 1) takes 27 bits of word 0 and 26 bits of word 1:
u = ((x0 >> 5) * 2**26 + (x1 >> 6)) * 2**-53.
"""

MASK32 = 0xFFFFFFFF
# Round multipliers and Weyl key increments of Philox4x32 (SC'11, Sec. 3.3).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85

PURPOSE_JUMP = 0


def _round(x, k):
    p0 = PHILOX_M0 * x[0]
    p1 = PHILOX_M1 * x[2]
    hi0, lo0 = p0 >> 32, p0 & MASK32
    hi1, lo1 = p1 >> 32, p1 & MASK32
    return (hi1 ^ x[1] ^ k[0], lo1, hi0 ^ x[3] ^ k[1], lo0)


def philox4x32_10(counter, key):
    """Ten Philox rounds; the key is bumped by the Weyl constants between rounds."""
    x = tuple(int(c) & MASK32 for c in counter)
    k = [int(key[0]) & MASK32, int(key[1]) & MASK32]
    for r in range(10):
        if r:
            k = [(k[0] + PHILOX_W0) & MASK32, (k[1] + PHILOX_W1) & MASK32]
        x = _round(x, k)
    return x


def uniform01(seed, traj, step, purpose=PURPOSE_JUMP):
    """Uniform double in [0, 1) for (seed, trajectory, step, purpose)."""
    seed = int(seed)
    step = int(step)
    x = philox4x32_10((traj, step & MASK32, purpose, (step >> 32) & MASK32),
                      (seed & MASK32, (seed >> 32) & MASK32))
    return ((x[0] >> 5) * 67108864 + (x[1] >> 6)) * (1.0 / 9007199254740992.0)
