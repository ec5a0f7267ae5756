"""Write twiddle_tables.cuh: roots of unity for the frame FFT kernels.

cos/sin of 2 pi k / N evaluated in double precision with Python's math module
and rounded to float32.  Run from this directory:  python gen_twiddles.py
"""
import math
import struct


def f32(v: float) -> str:
    r = struct.unpack("f", struct.pack("f", v))[0]
    s = repr(r)
    if "e" not in s and "." not in s:
        s += ".0"
    return s + "f"


def root(n: int, e: int):
    """exp(-2 pi i e / n) (forward sign) as (re, im) float32 literals."""
    a = 2.0 * math.pi * (e % n) / n
    return f32(math.cos(a)), f32(-math.sin(a))


def geometry(m: int):
    tx = m // 32
    tt = 32 // tx
    x0 = m // tt
    return tx, tt, x0


def main():
    out = ["// Generated by gen_twiddles.py -- do not edit.",
           "// Forward-sign roots of unity exp(-2 pi i e / N), float32.",
           "#pragma once", "", "namespace sharp {", ""]
    out.append("// cos(2 pi e / 32) and sin(2 pi e / 32), e in [0, 32)")
    for fn, trig in (("cos32", math.cos), ("sin32", math.sin)):
        out.append(f"__host__ __device__ __forceinline__ constexpr float {fn}(int e) {{")
        out.append("    switch (e & 31) {")
        for e in range(32):
            out.append(f"        case {e}: return {f32(trig(2 * math.pi * e / 32))};")
        out.append("    }")
        out.append("    return 0.0f;")
        out.append("}")
    out.append("")
    for m in (64, 128):
        tx, tt, x0 = geometry(m)
        vals = []
        for q in range(tx):
            for k in range(32):
                vals.append("{%s, %s}" % root(m, q * k))
        out.append(f"// tw1_{m}[q*32 + k] = W_{m}^(q k), q < {tx}")
        out.append(f"__constant__ float2 c_tw1_{m}[{tx * 32}] = {{" + ", ".join(vals) + "};")
        vals = []
        for a in range(x0):
            for t in range(tt):
                vals.append("{%s, %s}" % root(m, a * t))
        out.append(f"// tw2_{m}[x0*{tt} + t] = W_{m}^(x0 t), x0 < {x0}")
        out.append(f"__constant__ float2 c_tw2_{m}[{x0 * tt}] = {{" + ", ".join(vals) + "};")
        out.append("")
    vals = []
    for k in range(16):
        for j in range(16):
            vals.append("{%s, %s}" % root(256, j * k))
    out.append("// tw256x16[k*16 + j] = W_256^(j k), j, k < 16 (256 = 16 x 16 line transforms)")
    out.append("__constant__ float2 c_tw256x16[256] = {" + ", ".join(vals) + "};")
    out.append("")
    out.append("}  // namespace sharp")
    with open("twiddle_tables.cuh", "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
