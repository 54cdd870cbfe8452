"""Autotune the generic engine's tile shapes on this GPU and write the table.

    python -m paper_2405_02603_gb300.autotune [--out tuning/gb300.txt] [N ...]

Times every feasible (rows, columns) tile shape per (N, dtype) with
fsp_autotune (standalone solves), then tunes the mixed-size batched workload
(64 Vico-Greengard solves, N drawn with seed 2406 from {32,48,64,96,128,160})
with fsp_batch_autotune, whose shapes override those sizes, and writes the
table as "N dtype lgL_row lgL_col" lines.  The
table next to this file is loaded when the library is first used, which pins
the shapes (they change no result bit, only speed).  Default sizes: the
mixed-radix sizes of the batched and served workloads and the test sizes.
"""
import argparse
import os
import sys

DEFAULT_SIZES = [16, 24, 32, 40, 48, 60, 64, 80, 96, 120, 128, 160, 192, 240, 256]


def main(argv=None):
    here = os.path.dirname(os.path.abspath(__file__))
    ap = argparse.ArgumentParser()
    ap.add_argument("sizes", nargs="*", type=int)
    ap.add_argument("--out", default=os.path.join(here, "tuning", "gb300.txt"))
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(here))
    import paper_2405_02603_gb300 as fsp
    for N in args.sizes or DEFAULT_SIZES:
        for dtype in ("f64", "f32"):
            lr, lc = fsp.autotune(N, dtype)
            print("N=%d %s: rows 2^%d lines, columns 2^%d lines" % (N, dtype, lr, lc), flush=True)
    if not args.sizes:
        import numpy as np
        import torch
        Ns = [int(x) for x in np.random.default_rng(2406).choice([32, 48, 64, 96, 128, 160], size=64)]
        for dtype in ("f32", "f64"):
            plans = [fsp.Plan(N, 1.0, "vg_dct", dtype) for N in Ns]
            gen = torch.Generator(device="cuda").manual_seed(2406)
            rhos = [torch.rand((N, N, N), generator=gen, device="cuda", dtype=fsp.torch_dtype(dtype)) for N in Ns]
            phis = [torch.empty_like(r) for r in rhos]
            b = fsp.Batch(plans, rhos, phis)
            b.autotune()
            b.close()
            print("batch %s tuned" % dtype, flush=True)
    text = fsp.tuning_get()
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    with open(args.out, "w") as f:
        f.write(text)
    print(text)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
