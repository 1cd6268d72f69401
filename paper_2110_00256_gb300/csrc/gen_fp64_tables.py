"""Writes fp64_tables.h: the constants of the table-driven FP64 exponential and
logarithm in fp64_math.cuh (Tang's reductions), each correctly rounded to
double from a 200-bit evaluation with mpmath.  Run from this directory:

    python gen_fp64_tables.py > fp64_tables.h
"""
import mpmath as mp

mp.mp.prec = 200


def hexd(v) -> str:
    """Correctly rounded double of an mpmath number as a C hex-float literal."""
    return float(mp.mpf(v)).hex()


def split(v, bits):
    """v = hi + lo with hi keeping `bits` significant bits (hi * n exact for
    |n| < 2^(53 - bits)) and lo the correctly rounded rest."""
    v = mp.mpf(v)
    e = int(mp.floor(mp.log(abs(v), 2)))
    q = mp.mpf(2) ** (e - bits + 1)
    hi = mp.nint(v / q) * q
    return hi, v - hi


def main():
    ln2 = mp.log(2)
    out = ["// Generated by gen_fp64_tables.py (mpmath, 200 bits, each value correctly rounded"
           " to double).", "// Do not edit.", "#pragma once", ""]
    l_hi, l_lo = split(ln2 / 64, 32)
    n_hi, n_lo = split(ln2, 32)
    out += ["// exp: x = n ln2/64 + r, n = 64 k + j",
            f"constexpr double kExpInvL = {hexd(64 / ln2)};  // 64 / ln 2",
            f"constexpr double kExpLHi = {hexd(l_hi)};  // ln2/64, 32 bits",
            f"constexpr double kExpLLo = {hexd(l_lo)};",
            f"// log: ln x = e ln2 + ln c_j + log1p(r)",
            f"constexpr double kLn2Hi = {hexd(n_hi)};  // ln 2, 32 bits (e * kLn2Hi exact)",
            f"constexpr double kLn2Lo = {hexd(n_lo)};",
            ""]
    out.append("// 2^(j/64), j = 0 .. 63")
    out.append("__device__ const double kExp2J64[64] = {")
    vals = [hexd(mp.mpf(2) ** (mp.mpf(j) / 64)) for j in range(64)]
    out += ["    " + ", ".join(vals[i:i + 4]) + "," for i in range(0, 64, 4)]
    out.append("};")
    out.append("// c_j = 1 + (j + 1/2)/128 for j = 0 .. 63, (1 + (j + 1/2)/128)/2 for j = 64 .. 127")
    out.append("// (so that c_j lies in [0.75, 1.5)): 1/c_j and ln c_j, interleaved")
    out.append("__device__ const double kLogC128[256] = {")
    vals = []
    for j in range(128):
        c = 1 + (mp.mpf(j) + mp.mpf(1) / 2) / 128
        if j >= 64:
            c = c / 2
        vals += [hexd(1 / c), hexd(mp.log(c))]
    out += ["    " + ", ".join(vals[i:i + 4]) + "," for i in range(0, 256, 4)]
    out.append("};")
    print("\n".join(out))


if __name__ == "__main__":
    main()
