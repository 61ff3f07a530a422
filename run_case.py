"""Pack one named synthetic workload a few times through the C ABI.

A fixed, small driver for profilers (ncu) and quick checks:

    python run_case.py stars2k --reps 2
    python run_case.py batch --atlases 16 --reps 2
    python run_case.py pareto20k --reps 1 --check 3   # then the overlap counter


Exits non-zero if a pack fails.  Builds the library first if needed.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["plain64", "stars2k", "pareto20k", "batch"])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--atlases", type=int, default=16)
    ap.add_argument("--fanout", type=int, default=0)
    ap.add_argument("--direct", action="store_true",
                    help="launch the kernels directly (stage timing) instead of replaying the graph, whose "
                         "device-side wave loop profilers cannot enter")
    ap.add_argument("--check", type=int, default=0,
                    help="single-atlas cases: run the overlap and gutter counter this many times on the result")
    args = ap.parse_args(argv)

    import synth
    if args.case == "batch":
        sets = synth.stars_many(synth.batch256_specs(count=args.atlases))
    else:
        sets = [synth.WORKLOADS[args.case]()]

    from paper_2602_07782_gb300 import build, tabi
    build.build()
    need = sum(tabi.arena_bytes(cs) for cs in sets)
    ctx = tabi.Context(arena_bytes=min(need, 32 << 30) + (64 << 20))
    params = tabi.params_default(scale_fanout=args.fanout)
    if args.direct:
        ctx.stage_times(True)
    ks = None
    for _ in range(args.reps):
        if len(sets) == 1:
            r = ctx.pack(sets[0], params)
            res = [r]
        else:
            st, res = ctx.pack_batch(sets, params)
            if st != tabi.TABI_OK:
                print("batch failed:", tabi.status_str(st), ctx.last_error())
                return 1
        if any(r.status != tabi.TABI_OK for r in res):
            print("pack failed:", [tabi.status_str(r.status) for r in res], ctx.last_error())
            return 1
        ks = [r.k for r in res]
    print(args.case, "atlases", len(sets), "k", ks[:8], "..." if len(ks) > 8 else "")
    if args.check and len(sets) == 1:
        import numpy as np
        import torch
        cs, dev = sets[0], torch.device("cuda:0")
        offs = torch.from_numpy(cs.offsets.view(np.int32).copy()).to(dev)
        verts = torch.from_numpy(cs.verts.copy()).to(dev)
        place = torch.from_numpy(np.ascontiguousarray(res[0].place).view(np.uint8).copy()).to(dev)
        for _ in range(args.check):
            st, q = ctx.check_packing_device(cs.atlas_w, cs.atlas_h, params.gutter, cs.n, cs.nv, offs, verts, place)
            if st != tabi.TABI_OK or q != (0, 0, 0):
                print("check failed:", tabi.status_str(st), q, ctx.last_error())
                return 1
        print("overlap, gutter, outside texels:", q)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
