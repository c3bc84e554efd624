"""Counter-based random numbers for the LRS residual and the random-gamma mode.

Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): a 4 x 64-bit counter and a 2 x 64-bit key; each of 10 rounds
multiplies words 0 and 2 by fixed 64-bit constants, takes high/low halves of the
128-bit products and mixes them with words 1, 3 and the key; the key is bumped
by two Weyl constants between rounds.

Stream layout used by the LBM library (both sides implement it independently):
  key     = (seed, member)
  counter = (step, block, stream_id, 0), block = 0, 1, ... gives 4 words each
  stream_id 1 = LRS residual normals, 2 = random-gamma normals.

Normals come from Box-Muller on consecutive word pairs (2k, 2k+1):
  u1 = ((w_2k >> 11) + 1) 2^-53 in (0, 1],  u2 = (w_2k+1 >> 11) 2^-53 in [0, 1),
  z_2k = sqrt(-2 ln u1) cos(2 pi u2),  z_2k+1 = sqrt(-2 ln u1) sin(2 pi u2).
ln, cos and sin are this project's own series evaluations (below) using only
IEEE +, *, / and a correctly rounded sqrt, evaluated in a fixed order without
fused multiply-add, so that the normals are bit-reproducible on any IEEE
machine.
"""

import math

MASK64 = (1 << 64) - 1
_M0 = 0xD2E7470EE14C6C93
_M1 = 0xCA5A826395121157
_W0 = 0x9E3779B97F4A7C15   # golden ratio
_W1 = 0xBB67AE8584CAA73B   # sqrt(3) - 1

STREAM_LRS = 1
STREAM_GAMMA = 2

LN2 = 0.6931471805599453          # nearest double to ln 2
SQRT2 = 1.4142135623730951        # nearest double to sqrt 2
HALF_PI = 1.5707963267948966      # nearest double to pi / 2
_LOG_TERMS = 12                   # atanh series terms: s^(2k)/(2k+1), k < 12
_TRIG_TERMS = 13                  # Taylor terms for sin and cos on [0, pi/2)


def philox4x64_10(ctr, key):
    c0, c1, c2, c3 = (int(x) & MASK64 for x in ctr)
    k0, k1 = (int(x) & MASK64 for x in key)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        c0, c1, c2, c3 = ((p1 >> 64) ^ c1 ^ k0, p1 & MASK64, (p0 >> 64) ^ c3 ^ k1, p0 & MASK64)
        k0 = (k0 + _W0) & MASK64
        k1 = (k1 + _W1) & MASK64
    return [c0, c1, c2, c3]


def own_log(x):
    """ln x for a positive normal double: x = m 2^e with m in [sqrt2/2, sqrt2],
    ln x = e ln2 + 2 atanh(s), s = (m-1)/(m+1), atanh(s) = sum s^(2k+1)/(2k+1)
    (Horner in s^2, |s| <= 0.172)."""
    m, e = math.frexp(x)      # x = m 2^e, m in [0.5, 1)
    m = m * 2.0
    e = e - 1
    if m > SQRT2:
        m = m * 0.5
        e = e + 1
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    p = 1.0 / (2 * (_LOG_TERMS - 1) + 1)
    for k in range(_LOG_TERMS - 2, -1, -1):
        p = p * s2 + 1.0 / (2 * k + 1)
    t = s * p
    return float(e) * LN2 + (t + t)


def _inv_factorials(n):
    out = [1.0]
    for k in range(1, n):
        out.append(out[-1] / k)
    return out


_INVF = _inv_factorials(2 * _TRIG_TERMS + 2)


def own_cos_sin_2pi(u):
    """(cos 2 pi u, sin 2 pi u) for u in [0, 1) a multiple of 2^-53:
    4u = q + r exactly (quadrant q, r in [0, 1)), theta = r pi/2, Taylor series
    of cos and sin in theta (Horner in theta^2), then the quadrant rotation."""
    v = u * 4.0
    q = int(math.floor(v))
    r = v - q
    th = r * HALF_PI
    t2 = th * th
    cs = _INVF[2 * (_TRIG_TERMS - 1)] * (1 if (_TRIG_TERMS - 1) % 2 == 0 else -1)
    sn = _INVF[2 * (_TRIG_TERMS - 1) + 1] * (1 if (_TRIG_TERMS - 1) % 2 == 0 else -1)
    for k in range(_TRIG_TERMS - 2, -1, -1):
        sign = 1.0 if k % 2 == 0 else -1.0
        cs = cs * t2 + sign * _INVF[2 * k]
        sn = sn * t2 + sign * _INVF[2 * k + 1]
    sn = sn * th
    if q == 0:
        return cs, sn
    if q == 1:
        return -sn, cs
    if q == 2:
        return -cs, -sn
    return sn, -cs


def words(seed, member, step, stream, n):
    out = []
    block = 0
    while len(out) < n:
        out.extend(philox4x64_10((step, block, stream, 0), (seed, member)))
        block += 1
    return out[:n]


def normals(seed, member, step, stream, n):
    """n standard normals for (seed, member, step, stream), Box-Muller pairs."""
    npair = (n + 1) // 2
    w = words(seed, member, step, stream, 2 * npair)
    z = []
    for k in range(npair):
        u1 = ((w[2 * k] >> 11) + 1) * (1.0 / 9007199254740992.0)
        u2 = (w[2 * k + 1] >> 11) * (1.0 / 9007199254740992.0)
        r = math.sqrt(-2.0 * own_log(u1))
        c, s = own_cos_sin_2pi(u2)
        z.append(r * c)
        z.append(r * s)
    return z[:n]
