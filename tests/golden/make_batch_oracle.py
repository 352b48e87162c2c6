"""Write the FP64 oracle's DE fits of 8 sampled blocks of the 256-block batch.

The batch workload is synth.batch(0, nblocks=256): N log-uniform in 50K-1M
int16 samples, fs 1-50 kHz, pop 32-128, G = ceil(80000 / pop), each block with
its own Philox block id. Blocks 16, 48, ..., 240 (every 32nd) are fitted by
the CPU oracle alone, with the same draws as the batched GPU solve; the GPU
batch's fits of those blocks are compared with these. Calls only ``oracle``
and ``synth``. Fits are appended to batch_oracle_fits.json one at a time, so
an interrupted run keeps what it finished.

    python tests/golden/make_batch_oracle.py [--threads N]
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

OUT = os.path.join(HERE, "batch_oracle_fits.json")
SAMPLED = [16 + 32 * j for j in range(8)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    done = json.load(open(OUT)) if os.path.exists(OUT) else {}
    blocks = synth.batch(0, nblocks=256)
    for i in SAMPLED:
        key = str(i)
        if key in done:
            continue
        b = blocks[i]
        t = time.time()
        p, f = oracle.de_solve(b.values(), b.fs, b.t0, b.bounds, b.pop, b.gens, b.F, b.CR, b.de_seed,
                               block_id=b.block_id, nthreads=args.threads)
        done[key] = {"params": [float(v) for v in p], "sse": float(f),
                     "sse_truth": float(oracle.sse(b.values(), b.fs, b.t0, b.truth)),
                     "n": b.n, "fs": b.fs, "pop": b.pop, "gens": b.gens}
        with open(OUT, "w") as fh:
            json.dump(done, fh, indent=1, sort_keys=True)
        print(f"block {i}: n {b.n} pop {b.pop} gens {b.gens}: {time.time() - t:.0f} s", flush=True)


if __name__ == "__main__":
    main()
