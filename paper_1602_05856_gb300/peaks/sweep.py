"""Random-access rates of this GPU against buffer size (the roofline denominators).

    python -m paper_1602_05856_gb300.peaks.sweep            # 4 MiB .. 32 GiB, one line per size
    python -m paper_1602_05856_gb300.peaks.sweep --ncu-case # the two 32 MiB OR kernels, once each

Each line: log2 of the buffer's bytes, then random 64-bit atomic ORs and random
8-byte loads per second (G/s) with the 32-bit-LCG and the 64-bit-mixer address
streams of l2_random.cu. The --ncu-case run is small enough for an ncu capture.
"""
import argparse
import ctypes
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--ncu-case", action="store_true")
    p.add_argument("--lo", type=int, default=22)
    p.add_argument("--hi", type=int, default=35)
    args = p.parse_args()
    from paper_1602_05856_gb300 import build
    lib = ctypes.CDLL(build.build_peaks())
    f = lib.peaks_l2_random_rate
    f.restype = ctypes.c_double
    f.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
    if args.ncu_case:
        for mode, iters in ((1, 64), (4, 1024)):
            print(mode, f(mode, 32 << 20, iters, 1) / 1e9, flush=True)
        return
    for lg in range(args.lo, args.hi + 1):
        b = 1 << lg
        print(lg, json.dumps({"or_lcg": f(4, b, 1024, 3) / 1e9, "read_lcg": f(5, b, 1024, 3) / 1e9,
                              "or_mix": f(1, b, 64, 3) / 1e9, "read_mix": f(2, b, 64, 3) / 1e9}),
              flush=True)


if __name__ == "__main__":
    main()
