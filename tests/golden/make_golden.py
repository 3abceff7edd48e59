"""Write the oracle's expected values for the large, batched and served workloads.

Every number this script writes comes from ``oracle/`` (the plain binary64 CPU
implementation of Algorithm 1, Steps I-VII and Eqs. 6-7) on inputs from
``synthdata/``.  Nothing here touches the CUDA library.  The tests read the files
it writes and compare the GPU path against them field by field.

    python tests/golden/make_golden.py large          # 3 samples of n = 2^20
    python tests/golden/make_golden.py batch          # the 512-sample batch, n <= 65536
    python tests/golden/make_golden.py batch --all    # ... and the larger samples too
    python tests/golden/make_golden.py serve          # served stream, first 1000 requests, n <= 65536
    python tests/golden/make_golden.py serve_mid      # ... and those with 65536 < n <= 262144

Each line is written as soon as its sample is done, and a rerun skips the samples
already present, so a long run can be stopped and resumed.  The oracle's result
does not depend on its thread count (fixed row blocks, sums in row order).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(_HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthdata  # noqa: E402

FIELDS = ("mean", "sigma", "psi8", "g1", "psi6", "g2", "psi4", "h")
HEADER = "key n status " + " ".join(FIELDS)

FILES = {
    "large": "plugin_large_n1048576.txt",
    "batch": "plugin_batch512_seed6.txt",
    "serve": "plugin_serve1000_seed7_small.txt",
    "serve_mid": "plugin_serve1000_seed7_mid.txt",
}

DESCRIPTIONS = {
    "large": ("Oracle results (Algorithm 1, binary64, symmetric form of Eqs. 6-7) for the\n"
              "three n = 2^20 samples: Student-t3 seed 3, lognormal(0,1) seed 4, U[0,1] seed 5\n"
              "(synthdata.large_sample)."),
    "batch": ("Oracle results for the 512-sample batch (synthdata.batch_specs(512, 6, 256,\n"
              "262144)); key = sample index.  Samples with n <= 65536, and larger ones when\n"
              "written with --all."),
    "serve": ("Oracle results for the served stream (synthdata.server_specs(10000, 7, 1000,\n"
              "4194304)), binary32 samples widened to binary64; key = request index.  The\n"
              "first 1000 requests with n <= 65536."),
    "serve_mid": ("Oracle results for the served stream (synthdata.server_specs(10000, 7, 1000,\n"
                  "4194304)), binary32 samples widened to binary64; key = request index.  The\n"
                  "first 1000 requests with 65536 < n <= 262144."),
}


def _read_done(path: str) -> set[str]:
    done = set()
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                if line.strip() and not line.startswith("#"):
                    done.add(line.split()[0])
    return done


def _jobs(kind: str, include_all: bool):
    if kind == "large":
        for fam in ("t3", "lognormal", "uniform"):
            yield fam, (lambda fam=fam: synthdata.large_sample(fam))
    elif kind == "batch":
        for spec in synthdata.batch_specs(512, 6, 256, 262144):
            if include_all or spec.n <= 65536:
                yield str(spec.index), (lambda s=spec: synthdata.sample_from_spec(s))
    elif kind in ("serve", "serve_mid"):
        lo, hi = (0, 65536) if kind == "serve" else (65536, 262144)
        for spec in synthdata.server_specs(10000, 7, 1000, 4194304)[:1000]:
            if lo < spec.n <= hi:
                yield str(spec.index), (lambda s=spec: synthdata.sample_from_spec(s, np.float32)
                                        .astype(np.float64))
    else:
        raise ValueError(kind)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("kind", choices=sorted(FILES))
    ap.add_argument("--all", action="store_true", help="batch: include samples with n > 65536")
    ap.add_argument("--threads", type=int, default=None)
    args = ap.parse_args()
    path = os.path.join(_HERE, FILES[args.kind])
    done = _read_done(path)
    if not os.path.exists(path):
        with open(path, "w") as f:
            for line in DESCRIPTIONS[args.kind].splitlines():
                f.write(f"# {line}\n")
            f.write("# written by tests/golden/make_golden.py (oracle/ only)\n")
            f.write(f"# {HEADER}\n")
    for key, make in _jobs(args.kind, args.all):
        if key in done:
            continue
        x = make()
        t0 = time.time()
        res = oracle.plugin(x, threads=args.threads)
        vals = " ".join(f"{res[k]:.17g}" for k in FIELDS)
        with open(path, "a") as f:
            f.write(f"{key} {x.size} {res['status']} {vals}\n")
        print(f"{args.kind} {key} n={x.size} status={res['status']} h={res['h']:.17g} "
              f"{time.time() - t0:.1f}s", flush=True)


def load_file(kind: str) -> dict[str, dict]:
    """Parse one golden file into {key: {"n", "status", field: value}}."""
    out: dict[str, dict] = {}
    with open(os.path.join(_HERE, FILES[kind])) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            parts = line.split()
            rec = {"n": int(parts[1]), "status": int(parts[2])}
            rec.update({k: float(v) for k, v in zip(FIELDS, parts[3:])})
            out[parts[0]] = rec
    return out


def load(kind: str) -> dict[str, dict]:
    """The stored values of a workload: "serve" is the served stream's two files
    (n <= 65536, and 65536 < n <= 262144 where that file exists)."""
    out = load_file(kind)
    if kind == "serve" and os.path.exists(os.path.join(_HERE, FILES["serve_mid"])):
        out.update(load_file("serve_mid"))
    return out


if __name__ == "__main__":
    main()
