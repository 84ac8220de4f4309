"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
Random Numbers: As Easy as 1, 2, 3", SC'11), written from its published
definition.  The quantum-trajectory method needs one uniform number per
trajectory and time step to decide jump-or-evolve and pick the channel
(Sec. 4.1, jump probabilities W(alpha -> alpha^k) dt); drawing it from a
counter-based stream makes every (trajectory, step) draw independent of how the
work is scheduled.

Counter words: (trajectory id, step low 32 bits, purpose, step high 32 bits);
key words: (seed low 32 bits, seed high 32 bits).  Purpose 0 is the jump draw;
purpose 1 + j gives the j-th pair of Gaussian numbers of the quantum-state-
diffusion noise (Sec. 5.2).  A uniform double in [0, 1) takes 27 bits of one
word and 26 bits of the next: u = ((x0 >> 5) * 2**26 + (x1 >> 6)) * 2**-53.
"""
import math

MASK32 = 0xFFFFFFFF
# Round multipliers and Weyl key increments of Philox4x32 (SC'11, Sec. 3.3).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85

PURPOSE_JUMP = 0
PURPOSE_NOISE = 1  # the j-th Gaussian pair of a (trajectory, step) uses purpose 1 + j


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


def _draw(seed, traj, step, purpose):
    seed = int(seed)
    step = int(step)
    return philox4x32_10((traj, step & MASK32, purpose, (step >> 32) & MASK32),
                         (seed & MASK32, (seed >> 32) & MASK32))


def _uniform(hi, lo):
    return ((hi >> 5) * 67108864 + (lo >> 6)) * (1.0 / 9007199254740992.0)


def uniform01(seed, traj, step, purpose=PURPOSE_JUMP):
    """Uniform double in [0, 1) for (seed, trajectory, step, purpose)."""
    x = _draw(seed, traj, step, purpose)
    return _uniform(x[0], x[1])


def gaussian_pair(seed, traj, step, j):
    """The j-th pair of independent standard normal numbers of a (trajectory,
    step): the Box-Muller transform (Box and Muller, Ann. Math. Stat. 29, 1958)
    of the uniforms u1 (words 0, 1) and u2 (words 2, 3) of the draw with purpose
    PURPOSE_NOISE + j: r = sqrt(-2 ln(1 - u1)), phi = 2 pi u2, (r cos phi,
    r sin phi).  1 - u1 lies in (0, 1], so the logarithm is finite."""
    x = _draw(seed, traj, step, PURPOSE_NOISE + j)
    u1 = _uniform(x[0], x[1])
    u2 = _uniform(x[2], x[3])
    r = math.sqrt(-2.0 * math.log1p(-u1))
    phi = 2.0 * math.pi * u2
    return r * math.cos(phi), r * math.sin(phi)


def noise(seed, traj, step, n):
    """eta_k for k = 0 .. n-1: eta_{2j} and eta_{2j+1} are the j-th pair."""
    out = []
    for j in range((n + 1) // 2):
        out.extend(gaussian_pair(seed, traj, step, j))
    return out[:n]
