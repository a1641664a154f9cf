"""Writes twiddle128.h: exp(-2 pi i e / 128), e in [0, 128), from FP64 cos/sin,
as literal tables that the in-register transforms index with compile-time
indices (the values fold into the arithmetic instructions).
Run: python paper_2008_02478_gb300/csrc/gen_twiddles.py"""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    re = [math.cos(2 * math.pi * e / 128) for e in range(128)]
    im = [-math.sin(2 * math.pi * e / 128) for e in range(128)]
    fmt = lambda v: repr(float(v))
    lines = ["// Generated by gen_twiddles.py (FP64 cos/sin): w_128^e = exp(-2 pi i e / 128).",
             "#pragma once", "", "namespace boris {", ""]
    for name, vals in (("w128_re", re), ("w128_im", im)):
        lines.append("__host__ __device__ constexpr double %s(int e)" % name)
        lines.append("{")
        lines.append("    constexpr double t[128] = {")
        for i in range(0, 128, 4):
            lines.append("        " + ", ".join(fmt(v) for v in vals[i:i + 4]) + ",")
        lines.append("    };")
        lines.append("    return t[e];")
        lines.append("}")
        lines.append("")
    lines.append("}  // namespace boris")
    with open(os.path.join(HERE, "twiddle128.h"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
