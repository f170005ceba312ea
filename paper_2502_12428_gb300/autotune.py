"""Launch-shape autotuner: `python -m paper_2502_12428_gb300.autotune [--primes 3,5,7,11] [--what ring,sweep]`.

Per prime it times the fused engine on seeded random quartics and keeps the fastest candidate of two shapes:
- ring: the tile of the shared-memory slice ring that the int8 tensor form's chain runs over (work items per
  round x shared-memory ring size);
- sweep: the launch shape of the swept chain of the dp4a and int32 forms (the nonzero tap pairs from which a
  quartic runs every pair in the two-slice loop, and the CTAs per SM).  Its sample is half dense and half sparse
  quartics, since the threshold decides between the two paths only for quartics with zero coefficients.
It writes paper_2502_12428_gb300/tile_table.json, which the Python binding applies when it loads the library.
Heights do not depend on any of these shapes.
"""
import argparse
import json
import os
import sys

import numpy as np
import torch

from . import inputs
from . import qfs

DEFAULT_N = {3: 65536, 5: 32768, 7: 8192, 11: 512, 13: 128}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--primes", default="3,5,7,11")
    ap.add_argument("--quartics", type=int, default=0, help="sample size (default: sized per prime)")
    ap.add_argument("--out", default=qfs.TILE_TABLE)
    ap.add_argument("--what", default="ring,sweep", help="shapes to tune: ring, sweep or both")
    ap.add_argument("--sweep-forms", default="dp4a,int32")
    args = ap.parse_args(argv)
    what = set(args.what.split(","))
    table = {}
    if os.path.exists(args.out):
        with open(args.out) as fh:
            table = {int(k): v for k, v in json.load(fh).items()}
    for p in [int(x) for x in args.primes.split(",")]:
        n = args.quartics or DEFAULT_N[p]
        entry = table.get(p, {})
        if "ring" in what:
            sample = torch.from_numpy(inputs.dense(p, n, 0xA070 + p)).cuda()
            qfs.tune_set(p, 0, 0)
            best = qfs.autotune(p, sample, form="int8tc")
            best["quartics"] = n
            entry.update(best)
            print(json.dumps(best), flush=True)
        if "sweep" in what:
            half = max(1, n // 2)
            mix = np.concatenate([inputs.dense(p, half, 0xA170 + p), inputs.sparse(p, half, 0xA270 + p)])
            sample = torch.from_numpy(mix).cuda()
            sweeps = entry.get("sweep", {})
            for form in args.sweep_forms.split(","):
                qfs.sweep_tune_set(form, p, 0, 0)
                best = qfs.sweep_autotune(p, sample, form=form)
                best["quartics"] = int(sample.shape[0])
                sweeps[form] = best
                print(json.dumps({"p": p, "form": form, **best}), flush=True)
            entry["sweep"] = sweeps
        table[p] = entry
    qfs.save_tile_table(table, args.out)
    return 0


if __name__ == "__main__":
    sys.exit(main())
