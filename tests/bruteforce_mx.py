"""Exact-rational brute-force model of the MX-FFT for tiny transforms.

Written from the definitions, independently of the C oracle, for cross-checking
it on n0, n1 <= 8.  Every real number is a ``fractions.Fraction``; each FP32
operation is modelled as the exact result followed by one IEEE round-to-nearest-
even onto the binary32 grid (24-bit significand, subnormals down to 2^-149).
Twiddle components for n <= 8 are 0, +-1 or +-sqrt(2)/2; the irrational ones
are kept symbolic and quantised by comparing squares, so no approximation of
sqrt(2) enters.

Signs of zero are not modelled (Fractions have a single zero), so results are
compared by value.
"""
from __future__ import annotations

import math
from fractions import Fraction as Fr

import numpy as np

# OCP element formats: (mbits, emin, emax, maxnorm)
FORMATS = {
    "e4m3": (3, -6, 8, Fr(448)),
    "e5m2": (2, -14, 15, Fr(57344)),
    "e2m3": (3, 0, 2, Fr(15, 2)),
    "e3m2": (2, -2, 4, Fr(28)),
    "e2m1": (1, 0, 2, Fr(6)),
}


def floor_log2(x: Fr) -> int:
    """floor(log2 x) for a positive rational."""
    e = x.numerator.bit_length() - x.denominator.bit_length()
    while Fr(2) ** e > x:
        e -= 1
    while Fr(2) ** (e + 1) <= x:
        e += 1
    return e


def round_half_even(n: Fr) -> int:
    f = math.floor(n)
    d = n - f
    if d > Fr(1, 2) or (d == Fr(1, 2) and f % 2 == 1):
        f += 1
    return f


def f32(x: Fr) -> Fr:
    """Round an exact rational to the nearest binary32 value (ties to even)."""
    if x == 0:
        return Fr(0)
    s = 1 if x > 0 else -1
    a = abs(x)
    E = max(floor_log2(a), -126)
    q = Fr(2) ** (E - 23)
    r = round_half_even(a / q) * q
    if r >= Fr(2) ** 128:
        raise OverflowError("binary32 overflow")
    return s * r


def f32_sqrt(s: Fr) -> Fr:
    """Correctly rounded binary32 square root of a positive rational."""
    E = max(floor_log2(s) // 2, -126)
    q = Fr(2) ** (E - 23)
    z = s / (q * q)  # want round(sqrt(z))
    f = math.isqrt(z.numerator * z.denominator) // z.denominator
    mid = (Fr(f) + Fr(1, 2)) ** 2
    if z > mid or (z == mid and f % 2 == 1):
        f += 1
    return f * q


def ldexp32(x: Fr, e: int) -> Fr:
    return f32(x * Fr(2) ** e)


class Surd:
    """c * sqrt(2) with c rational (only the twiddle components +-sqrt(2)/2)."""

    def __init__(self, c: Fr):
        self.c = Fr(c)

    def sq(self) -> Fr:
        return 2 * self.c * self.c


def _abs_sq(v) -> Fr:
    return v.sq() if isinstance(v, Surd) else Fr(v) * Fr(v)


def q_elem(x, fmt: str) -> Fr:
    """Nearest element-grid value (ties to even), saturating, for a rational
    or a Surd argument."""
    mbits, emin, emax, maxn = FORMATS[fmt]
    if isinstance(x, Surd):
        if x.c == 0:
            return Fr(0)
        sgn = 1 if x.c > 0 else -1
        a2 = x.sq()                       # |x|^2, rational
        E = max(floor_log2(a2) // 2, emin)
        q = Fr(2) ** (E - mbits)
        z = a2 / (q * q)                  # (|x|/q)^2
        f = math.isqrt(z.numerator * z.denominator) // z.denominator
        if z > (Fr(f) + Fr(1, 2)) ** 2:   # never a tie: |x|/q is irrational
            f += 1
        r = min(f * q, maxn)
        return sgn * r
    x = Fr(x)
    if x == 0:
        return Fr(0)
    sgn = 1 if x > 0 else -1
    a = abs(x)
    E = max(floor_log2(a), emin)
    q = Fr(2) ** (E - mbits)
    r = min(round_half_even(a / q) * q, maxn)
    return sgn * r


def scale_exp(amax_sq: Fr, fmt: str) -> int:
    """Shared exponent from the squared block maximum (E8M0 range)."""
    if amax_sq == 0:
        return 0
    _, _, emax, _ = FORMATS[fmt]
    return min(max(floor_log2(amax_sq) // 2 - emax, -127), 127)


def twiddle(j: int, h: int, inverse: bool):
    """exp(-+ i pi j / h) for h <= 4 as (re, im), exact or Surd."""
    eighth = (8 * j) // (2 * h) if (8 * j) % (2 * h) == 0 else None
    assert eighth is not None, "only multiples of pi/4"
    r2 = Surd(Fr(1, 2))
    table = {0: (1, 0), 1: (r2, Surd(Fr(1, 2))), 2: (0, 1), 3: (Surd(Fr(-1, 2)), Surd(Fr(1, 2))),
             4: (-1, 0)}
    re, im = table[eighth]
    # exp(-i a) = cos a - i sin a for the forward transform
    if not inverse:
        im = Surd(-im.c) if isinstance(im, Surd) else -im
    return re, im


def _mul_pow2(v, e: int):
    return Surd(v.c * Fr(2) ** e) if isinstance(v, Surd) else Fr(v) * Fr(2) ** e


def butterfly_block(U, V, W, fmt):
    """Alg. 2 on one block.  U, V: lists of (re, im) binary32 rationals;
    W: list of (re, im) exact twiddles.  Returns (Y0, Y1)."""
    mbits, emin, emax, maxn = FORMATS[fmt]
    aw2 = max(max(_abs_sq(w[0]), _abs_sq(w[1])) for w in W)
    sw = scale_exp(aw2, fmt)
    X = [(q_elem(_mul_pow2(w[0], -sw), fmt), q_elem(_mul_pow2(w[1], -sw), fmt)) for w in W]
    av = max(max(abs(v[0]), abs(v[1])) for v in V)
    sv = scale_exp(av * av, fmt)
    Y = [(q_elem(ldexp32(v[0], -sv), fmt), q_elem(ldexp32(v[1], -sv), fmt)) for v in V]
    P = []
    for (xr, xi), (yr, yi) in zip(X, Y):
        pr = f32(f32(xr * yr) - f32(xi * yi))
        pi = f32(f32(xr * yi) + f32(xi * yr))
        P.append((pr, pi))
    sout = sw + sv
    pmax = max(max(abs(p[0]), abs(p[1])) for p in P)
    if pmax > maxn:  # renormalisation: smallest r with pmax <= maxn 2^r
        r = 0
        while pmax > maxn * Fr(2) ** r:
            r += 1
        P = [(ldexp32(p[0], -r), ldexp32(p[1], -r)) for p in P]
        sout += r
        pmax = pmax / Fr(2) ** r
    if pmax == 0:
        shat = sout
    else:
        shat = min(max(sout + floor_log2(pmax) - emax, -127), 127)
    Y0, Y1 = [], []
    for (u, p) in zip(U, P):
        c = (q_elem(ldexp32(p[0], sout - shat), fmt), q_elem(ldexp32(p[1], sout - shat), fmt))
        wv = (ldexp32(c[0], shat), ldexp32(c[1], shat))
        Y0.append((f32(u[0] + wv[0]), f32(u[1] + wv[1])))
        Y1.append((f32(u[0] - wv[0]), f32(u[1] - wv[1])))
    return Y0, Y1


def bitrev(i: int, bits: int) -> int:
    return int(format(i, f"0{bits}b")[::-1], 2) if bits else 0


def fft1d(A, kblk: int, fmt: str, inverse: bool):
    n = len(A)
    L = n.bit_length() - 1
    A = _bitrev_perm(A, L)
    m = min(kblk // 2, n // 2)
    h = 1
    while h < n:
        order = []
        for b in range(n // 2):
            g, j = divmod(b, h)
            order.append((2 * h * g + j, 2 * h * g + j + h, j))
        for beta in range(len(order) // m):
            blk = order[beta * m:(beta + 1) * m]
            U = [A[iu] for iu, _, _ in blk]
            V = [A[iv] for _, iv, _ in blk]
            W = [twiddle(j, h, inverse) for _, _, j in blk]
            Y0, Y1 = butterfly_block(U, V, W, fmt)
            for (iu, iv, _), y0, y1 in zip(blk, Y0, Y1):
                A[iu] = y0
                A[iv] = y1
        h *= 2
    return A


def _bitrev_perm(A, L):
    out = [None] * len(A)
    for i, a in enumerate(A):
        out[bitrev(i, L)] = a
    return out


def magnitude(re: Fr, im: Fr) -> Fr:
    if re == 0 and im == 0:
        return Fr(0)
    e = max(floor_log2(abs(c)) + 1 for c in (re, im) if c != 0)  # frexp exponent
    a = ldexp32(re, -e)
    b = ldexp32(im, -e)
    s = f32(f32(a * a) + f32(b * b))
    return ldexp32(f32_sqrt(s), e)


def prescale_k(S, tau32: Fr, target: Fr, tau_min: Fr, kmin=-126, kmax=126) -> int:
    mags = [magnitude(re, im) for row in S for (re, im) in row]
    amax = max(mags)
    if amax == 0:
        return 0
    nz = sorted(m for m in mags if m > 0)
    r = math.floor(f32(tau32 * f32(Fr(len(nz) - 1))))
    p = nz[r]
    eps = Fr(1e-30)
    z = (target / max(amax, eps)) ** 2       # k1 = round(log2 sqrt(z))
    L = floor_log2(z)
    k1 = (L + 1) // 2
    y = tau_min / max(p, eps)                 # k2 = ceil(log2 y)
    Ly = floor_log2(y)
    k2 = Ly if Fr(2) ** Ly == y else Ly + 1
    return min(max(max(k1, k2), kmin), kmax)


def _rows(S, kblk, fmt, inverse):
    return [fft1d(list(row), kblk, fmt, inverse) for row in S]


def _cols(S, kblk, fmt, inverse):
    n0, n1 = len(S), len(S[0])
    S = [list(row) for row in S]
    for c in range(n1):
        col = fft1d([S[r][c] for r in range(n0)], kblk, fmt, inverse)
        for r in range(n0):
            S[r][c] = col[r]
    return S


def _transform2d(S, kblk, fmt, inverse):
    return _cols(_rows(S, kblk, fmt, inverse), kblk, fmt, inverse)


def mxfft2d(x: np.ndarray, fmt: str, kblk: int, op: str = "forward", tau=1e-3,
            target=Fr(1, 2), tau_min=None, kmin=-126, kmax=126):
    """One complex64 slice [n0, n1] -> (complex128 result, k or (k, k_inv))."""
    if tau_min is None:
        tau_min = Fr(1, 4096) if fmt == "e5m2" else Fr(1, 1024)
    tau32 = Fr(float(np.float32(tau)))
    S = [[(Fr(float(z.real)), Fr(float(z.imag))) for z in row] for row in np.asarray(x, np.complex64)]
    k = prescale_k(S, tau32, Fr(target), Fr(tau_min), kmin, kmax)
    S = [[(ldexp32(a, k), ldexp32(b, k)) for (a, b) in row] for row in S]
    S = _transform2d(S, kblk, fmt, inverse=(op == "inverse"))
    lg = (len(S).bit_length() - 1) + (len(S[0]).bit_length() - 1)
    if op == "roundtrip_fused":
        # encode once, F, then F^-1 columns first on the undecoded result,
        # decode once
        S = _rows(_cols(S, kblk, fmt, True), kblk, fmt, True)
        S = [[(ldexp32(a, -k - lg), ldexp32(b, -k - lg)) for (a, b) in row] for row in S]
        out = np.array([[complex(float(a), float(b)) for (a, b) in row] for row in S])
        return out, k
    S = [[(ldexp32(a, -k), ldexp32(b, -k)) for (a, b) in row] for row in S]
    kout = k
    if op == "roundtrip":
        kinv = prescale_k(S, tau32, Fr(target), Fr(tau_min), kmin, kmax)
        S = [[(ldexp32(a, kinv), ldexp32(b, kinv)) for (a, b) in row] for row in S]
        S = _transform2d(S, kblk, fmt, inverse=True)
        S = [[(ldexp32(a, -kinv - lg), ldexp32(b, -kinv - lg)) for (a, b) in row] for row in S]
        kout = (k, kinv)
    out = np.array([[complex(float(a), float(b)) for (a, b) in row] for row in S])
    return out, kout
