"""Chain tile autotuner: `python -m paper_2502_12428_gb300.autotune [--primes 3,5,7,11] [--quartics N]`.

For every prime it times the fused engine on seeded random quartics for each candidate tile shape (work items per
round x shared-memory ring size) of the shared-memory slice ring, which the int8 tensor form's chain runs over (the
dp4a and int32 forms sweep the slices from global memory and have no tile).  It keeps the fastest and writes the
table to paper_2502_12428_gb300/tile_table.json, which the Python binding applies when it loads the library.
Heights do not depend on the tile shape.
"""
import argparse
import json
import sys

import torch

from . import inputs
from . import qfs


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--primes", default="3,5,7,11")
    ap.add_argument("--quartics", type=int, default=0, help="sample size (default: sized per prime)")
    ap.add_argument("--out", default=qfs.TILE_TABLE)
    ap.add_argument("--form", default="int8tc", choices=sorted(qfs.FORMS))
    args = ap.parse_args(argv)
    default_n = {3: 65536, 5: 32768, 7: 8192, 11: 512, 13: 128}
    table = {}
    for p in [int(x) for x in args.primes.split(",")]:
        n = args.quartics or default_n[p]
        sample = torch.from_numpy(inputs.dense(p, n, 0xA070 + p)).cuda()
        qfs.tune_set(p, 0, 0)
        best = qfs.autotune(p, sample, form=args.form)
        best["quartics"] = n
        table[p] = best
        print(json.dumps(best), flush=True)
    qfs.save_tile_table(table, args.out)
    return 0


if __name__ == "__main__":
    sys.exit(main())
