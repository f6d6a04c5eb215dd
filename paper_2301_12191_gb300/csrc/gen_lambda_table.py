"""Writes lambda_table.inc: the frozen integer lambda table of the CUDA path.

lambda_Q16[qp] = round(65536 * sqrt(0.57 * 2^((qp - 12) / 3))), qp = 0..51.
The paper gives no lambda; this is the SAD-domain lambda of common HEVC
encoders.  The kernels use only the integer table, so every decision stays
integer.  Run once; the output is committed.
"""
import math
import os

vals = [int(math.floor(65536.0 * math.sqrt(0.57 * 2.0 ** ((qp - 12) / 3.0)) + 0.5)) for qp in range(52)]
out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lambda_table.inc")
with open(out, "w") as f:
    f.write("/* generated by gen_lambda_table.py: round(65536*sqrt(0.57*2^((qp-12)/3))) */\n")
    for i in range(0, 52, 6):
        f.write("    " + ", ".join(f"{v}" for v in vals[i:i + 6]) + ",\n")
print(out)
