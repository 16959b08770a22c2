"""Tables for the double-float (FP32 pair) logarithm and sine/cosine.

Written at build time into the generated header dfloat_tables.h.  Values are
computed with Python's decimal module at 60 digits and split into
(hi, lo) = (fl32(v), fl32(v - hi)), so hi + lo carries about 48 bits.

  log table (Tang's table-driven method, ACM TOMS 16 (1990) 378): for
  j = 0..127, m_j = 1 + (j + 1/2)/128, c_j = fl32(1/m_j) and L_j = -ln(c_j)
  (exact logarithm of the float c_j), so log(m) = L_j + log1p(m c_j - 1).
  sine/cosine table: cos(pi j/128), sin(pi j/128) for j = 0..256.
"""
from decimal import Decimal, getcontext

import numpy as np

getcontext().prec = 60


def _pi():
    # Machin: pi = 16 atan(1/5) - 4 atan(1/239)
    def atan_inv(x):
        x = Decimal(x)
        term = 1 / x
        s = term
        x2 = x * x
        k = 1
        while True:
            term = term / x2
            t = term / (2 * k + 1)
            if t == 0 or abs(t) < Decimal(10) ** -70:
                break
            s += -t if k % 2 else t
            k += 1
        return s
    return 16 * atan_inv(5) - 4 * atan_inv(239)


PI = _pi()


def _sin_cos(x):
    s, c = Decimal(0), Decimal(0)
    term = Decimal(1)
    k = 0
    while True:
        if k > 0:
            term = term * x / k
        if abs(term) < Decimal(10) ** -70:
            break
        r = k % 4
        if r == 0:
            c += term
        elif r == 1:
            s += term
        elif r == 2:
            c -= term
        else:
            s -= term
        k += 1
    return s, c


def split(v):
    hi = np.float32(float(v))
    lo = np.float32(float(v - Decimal(float(hi))))
    return float(hi), float(lo)


def _f(x):
    return repr(float(np.float32(x))) + "f"


def header():
    lines = ["// Generated by paper_1305_0708_gb300.compiler.dftables (decimal, 60 digits).", "#pragma once",
             "#ifdef __CUDA_ARCH__", "#define ME_TAB(name) name##_d", "#else", "#define ME_TAB(name) name##_h",
             "#endif", "namespace me {"]

    def arr(nm, vals):
        body = ", ".join(_f(x) for x in vals)
        lines.append(f"__device__ const float {nm}_d[{len(vals)}] = {{{body}}};")
        lines.append(f"static const float {nm}_h[{len(vals)}] = {{{body}}};")
    c, Lhi, Llo = [], [], []
    for j in range(128):
        mj = 1 + (Decimal(j) + Decimal("0.5")) / 128
        cj = np.float32(float(1 / mj))
        L = -Decimal(float(cj)).ln()
        hi, lo = split(L)
        c.append(float(cj))
        Lhi.append(hi)
        Llo.append(lo)
    arr("kLogC", c)
    arr("kLogLhi", Lhi)
    arr("kLogLlo", Llo)
    ch, cl, sh, sl = [], [], [], []
    for j in range(257):
        s, co = _sin_cos(PI * j / 128)
        a, b = split(co)
        ch.append(a)
        cl.append(b)
        a, b = split(s)
        sh.append(a)
        sl.append(b)
    for nm, vals in (("kCosHi", ch), ("kCosLo", cl), ("kSinHi", sh), ("kSinLo", sl)):
        arr(nm, vals)
    ln2 = Decimal(2).ln()
    lines.append("constexpr float kLn2Hi = %s, kLn2Lo = %s;" % tuple(_f(x) for x in split(ln2)))
    lines.append("constexpr float kPiHi = %s, kPiLo = %s;" % tuple(_f(x) for x in split(PI)))
    lines.append("constexpr float kInvPiHi = %s, kInvPiLo = %s;" % tuple(_f(x) for x in split(1 / PI)))
    lines.append("constexpr float kInv2PiHi = %s, kInv2PiLo = %s;" % tuple(_f(x) for x in split(1 / (2 * PI))))
    lines.append("constexpr float kInv4PiHi = %s, kInv4PiLo = %s;" % tuple(_f(x) for x in split(1 / (4 * PI))))
    lines.append("constexpr float kThirdHi = %s, kThirdLo = %s;" % tuple(_f(x) for x in split(Decimal(1) / 3)))
    lines.append("constexpr float kSixthHi = %s, kSixthLo = %s;" % tuple(_f(x) for x in split(Decimal(1) / 6)))
    lines.append("}  // namespace me")
    return "\n".join(lines) + "\n"
