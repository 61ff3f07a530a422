"""Time and scale of the packer under the paper's ablation settings, on the
synthetic workloads (the paper's chart sets are not available).

    python ablate.py [--reps 20] [--json out.json]

Three studies, each on one GPU, one atlas per pack through tabi_pack_device
(inputs resident), the pack time the median of --reps packs after warm-up
(CUDA events on the packing stream), the scale k*/1024 and the L^2 stretch
1024/k* (Sec. 5: one common scale s gives stretch 1/s):

  * t_opt (Sec. 4.4, Tab. 4): the prefix-sum tail at 0, 1, 2 and 5 % of the
    atlas height on the 20,000-chart Pareto workload (4096^2);
  * the local-AABB count (Tab. 13): 2, 5 and 10 slices per axis on the
    2,000-star workload (2048^2);
  * tightness and balance (Tab. 3): the full method, tight only (no
    direction choice or knees), balanced only (bounding boxes, no
    compaction) and the Chameleon-like baseline (boxes, static alternation)
    on the 2,000-star and the knees workloads.

Every setting measured here is one the GPU parity tests compare with the
CPU oracle (tests/test_gpu_parity.py: the ablation flags, the local-AABB
counts and the prefix-sum tail); this driver only times them.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _time_pack(ctx, cs, params, reps, torch, tabi, dev, stream):
    import numpy as np
    offs = torch.from_numpy(cs.offsets.view(np.int32).copy()).to(dev)
    verts = torch.from_numpy(cs.verts.copy()).to(dev)
    out = torch.zeros(tabi.PLACEMENT_DTYPE.itemsize * cs.n, dtype=torch.uint8, device=dev)
    ms, k = [], None
    for i in range(reps + 3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            st, k = ctx.pack_device(cs.n, cs.nv, cs.atlas_w, cs.atlas_h, offs, verts, out, params, stream=stream)
            b.record(stream)
        if st != tabi.TABI_OK:
            raise RuntimeError(f"pack failed: {tabi.status_str(st)} {ctx.last_error()}")
        b.synchronize()
        if i >= 3:
            ms.append(a.elapsed_time(b))
    return float(np.median(ms)), int(k)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)

    import torch

    import synth
    from paper_2602_07782_gb300 import build, tabi
    build.build()
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(device=dev)
    work = {"pareto20k": synth.pareto20k(), "stars2k": synth.stars2k(), "knees2k": synth.knees(11, 2000, 2048)}
    ctx = tabi.Context(arena_bytes=max(tabi.arena_bytes(cs) for cs in work.values()) + (256 << 20))
    F = tabi
    studies = []
    for topt in (0, 10, 20, 50):
        studies.append(("t_opt", f"{topt / 10:g} %", "pareto20k", dict(topt_permille=topt)))
    for kk in (2, 5, 10):
        studies.append(("local AABBs", str(kk), "stars2k", dict(laabb_count=kk)))
    for name in ("stars2k", "knees2k"):
        for label, flags in (("full", F.F_ALL), ("tight only", F.F_ALL & ~F.F_BALANCE),
                             ("balanced only", F.F_BALANCE), ("boxes, alternation", 0)):
            studies.append(("tight / balanced", label, name, dict(flags=flags)))
    rows = []
    for study, setting, name, kw in studies:
        cs = work[name]
        p = tabi.params_default(**kw)
        ms, k = _time_pack(ctx, cs, p, args.reps, torch, tabi, dev, stream)
        row = {"study": study, "setting": setting, "workload": name, "charts": cs.n,
               "atlas": f"{cs.atlas_w}x{cs.atlas_h}", "ms": round(ms, 3), "k": k,
               "stretch": round(1024.0 / k, 4)}
        rows.append(row)
        print(json.dumps(row), flush=True)
    ctx.close()
    if args.json:
        with open(args.json, "w") as f:
            json.dump(rows, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
