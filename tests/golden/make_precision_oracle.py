"""Write the FP64 oracle's DE fits of the precision-sweep blocks.

For each seed and sample storage, the paper-size block (N = 400,000 at
10 kHz, pop 64, 1250 generations, F 0.7, CR 0.9) is fitted by the CPU
oracle alone; the GPU tiers' fits are compared with these. Calls only
``oracle`` and ``synth``. Results are appended to precision_oracle_fits.json
one fit at a time, so an interrupted run keeps what it finished.

    python tests/golden/make_precision_oracle.py [--seeds 32] [--threads N]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(HERE, "precision_oracle_fits.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=32)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--storages", default="i8,f16,f32")
    args = ap.parse_args()
    done = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for seed in range(args.seeds):
        for st in args.storages.split(","):
            key = f"{st}/{seed}"
            if key in done:
                continue
            b = synth.precision(seed, synth.STORAGE_NAMES[st])
            t = time.time()
            p, f = oracle.de_solve(b.values(), b.fs, b.t0, b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed,
                                   nthreads=args.threads)
            done[key] = {"params": [float(v) for v in p], "sse": f, "truth": [float(v) for v in b.truth],
                         "sse_truth": oracle.sse(b.values(), b.fs, b.t0, b.truth), "seconds": time.time() - t}
            tmp = OUT + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(done, fh, indent=0, sort_keys=True)
            os.replace(tmp, OUT)
            print(key, f"{time.time() - t:.1f}s", flush=True)


if __name__ == "__main__":
    main()
