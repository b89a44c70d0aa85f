"""Write tests/golden/oracle_vectors.txt from the CPU oracle alone.

The SparkCL paper prints no worked numeric example, so these are regression
vectors of the (separately pinned) oracle: a change to the oracle's arithmetic
shows up as a diff here.  Run: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

MIX_INPUTS = [0, 1, 2, 3, 0xFFFFFFFF, 0x12345678, 0x80000000, 0xDEADBEEF]
POLY_INPUTS = [0.0, 1.0, -1.0, 2.0, -2.0, 0.5, 3.0, -0.1, 1e-3, 7.25]


def main():
    lines = ["# oracle regression vectors (written by make_golden.py, oracle only)",
             "# mix32 <x hex> <mix32(x) hex>",
             "# poly3 <x f32 bits hex> <poly3(x) f32 bits hex>  coef {0.5f, -1.25f, 0.1f}",
             "# mix32_sum_range <lo> <hi> <sum of mix32 over [lo, hi)>"]
    for x in MIX_INPUTS:
        lines.append("mix32 %08x %08x" % (x, oracle.mix32(x)))
    for x in POLY_INPUTS:
        xf = np.float32(x)
        y = oracle.poly3(xf)
        lines.append("poly3 %08x %08x" % (int(xf.view(np.uint32)),
                                          int(np.float32(y).view(np.uint32))))
    for lo, hi in ((0, 1024), (0, 1 << 20), (123_456, 7_654_321)):
        lines.append("mix32_sum_range %d %d %d" % (lo, hi, oracle.mix32_sum_range(lo, hi)))
    with open(os.path.join(HERE, "oracle_vectors.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
