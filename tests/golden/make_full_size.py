"""Write the full-size expected values of the resultant workloads.

    python tests/golden/make_full_size.py [--threads N] [--only NAME[,NAME]] [--o1-seconds S] [--o1-only]

Every expected value here comes from ``oracle/`` alone: the independent
modular oracle O2 (``oracle.modular``) computes each resultant exactly, and
its SHA-256 digest over the canonical text of the coefficient list
(``oracle.modular.digest``), the degree and the largest coefficient's bit
length are stored in ``full_size.json``.  Inputs come from the seeded
generators of ``paper_1010_1386_gb300.inputs`` (layout only, no resultant
arithmetic), the same ones the GPU tests draw.  ``--o1-seconds`` also runs
the exact oracle O1 (``oracle.exact``, Kronecker map + integer Bareiss) on
the smallest instances of each workload for up to that many seconds per
workload and stores its digests in ``o1_pins.json``, which the CPU tests use
to pin O2 to O1 at sizes too large to recompute there.
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import exact, modular  # noqa: E402
from paper_1010_1386_gb300 import inputs  # noqa: E402

ENCODING = ("sha256 of the text '<degree>;' followed by every coefficient of R, low to high, in signed "
            "hexadecimal without prefix, comma-separated (Python format(c, 'x')); degree -1 and no "
            "coefficients for R = 0")


def _swap(p):
    """The same polynomial with x and y exchanged (limb array layout)."""
    return np.ascontiguousarray(p.coeffs.transpose(1, 0, 2))


def workloads():
    """name -> (description, zero-argument function returning the pairs)."""
    def shift(deg, sparse, k):
        def make():
            base = inputs.workload_shift(5, deg, sparse, k)
            return [(f.coeffs, g.coeffs) for f, g in base] + [(_swap(f), _swap(g)) for f, g in base]
        return (f"shift workload, total degree {deg}, {'sparse' if sparse else 'dense'}, k = {k}: "
                f"Res_y of the 10 pairs of inputs.workload_shift(5, {deg}, {sparse}, {k}), then Res_x "
                f"(Res_y with x and y exchanged) of the same pairs"), make
    return {
        "c0_small": ("inputs.workload_small(0): one pair, dense total degree 6, coefficients in [-2^10, 2^10]",
                     lambda: inputs.workload_small(0)),
        "c1_single": ("inputs.workload_single(1): one pair, dense total degree 30, signed 32-bit",
                      lambda: inputs.workload_single(1)),
        "c2_batch": ("inputs.workload_batch(2, n=512): 512 pairs, deg_x, deg_y ~ U[8, 40], bits in {16, 32, 64}",
                     lambda: inputs.workload_batch(2, n=512)),
        "c3_nongeneric": ("inputs.workload_nongeneric(3, n=32): f = p q^2, g = df/dy (R = 0)",
                          lambda: inputs.workload_nongeneric(3, n=32)),
        "c3p_nongeneric_coprime": ("inputs.workload_nongeneric(3, n=32, coprime=True): f = p q^2, g = d(pq)/dy",
                                   lambda: inputs.workload_nongeneric(3, n=32, coprime=True)),
        "c4_serving_first512": ("the first 512 requests of inputs.workload_serving(4, n=10000)",
                                lambda: inputs.workload_serving(4, n=512)[0]),
        "shift_9_dense_128": shift(9, False, 128),
        "shift_9_sparse_2048": shift(9, True, 2048),
        "shift_15_dense_512": shift(15, False, 512),
        "shift_15_dense_2048": shift(15, False, 2048),
    }


def record(R):
    return {"deg": len(R) - 1, "bits": max((abs(c).bit_length() for c in R), default=0),
            "sha256": modular.digest(R)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    ap.add_argument("--only", default=None)
    ap.add_argument("--o1-seconds", type=float, default=0.0)
    ap.add_argument("--o1-only", action="store_true", help="skip O2; only add O1 digests")
    args = ap.parse_args()
    path = os.path.join(HERE, "full_size.json")
    data = json.load(open(path)) if os.path.exists(path) else {}
    data["encoding"] = ENCODING
    data["oracle"] = "oracle/modres.c (O2) through oracle/modular.py"
    data.setdefault("workloads", {})
    names = args.only.split(",") if args.only else list(workloads())
    for name in ([] if args.o1_only else names):
        desc, make = workloads()[name]
        pairs = make()
        t = time.time()
        rs = modular.resultants(pairs, threads=args.threads)
        dt = time.time() - t
        data["workloads"][name] = {"inputs": desc, "seconds": round(dt, 1), "threads": args.threads,
                                   "results": [record(R) for R in rs]}
        print(f"{name}: {len(rs)} resultants in {dt:.1f} s", flush=True)
        with open(path, "w") as fh:
            json.dump(data, fh, indent=0, sort_keys=True)
            fh.write("\n")
    if args.o1_seconds > 0:
        o1_path = os.path.join(HERE, "o1_pins.json")
        o1 = json.load(open(o1_path)) if os.path.exists(o1_path) else {}
        o1["encoding"] = ENCODING
        o1["oracle"] = "oracle/exact.py resultant_y (O1: Kronecker map x -> 2^k, integer Bareiss)"
        o1.setdefault("workloads", {})
        for name in names:
            _, make = workloads()[name]
            pairs = make()
            arr = [(modular.limbs_array(f), modular.limbs_array(g)) for f, g in pairs]
            size = [a.shape[0] * a.shape[1] * a.shape[2] + b.shape[0] * b.shape[1] * b.shape[2] for a, b in arr]
            order = sorted(range(len(pairs)), key=lambda i: size[i])
            done = o1["workloads"].setdefault(name, {})
            t0 = time.time()
            for i in order:
                if time.time() - t0 > args.o1_seconds:
                    break
                if str(i) in done:
                    continue
                a, b = arr[i]
                F = [[_int(a[x, y]) for y in range(a.shape[1])] for x in range(a.shape[0])]
                G = [[_int(b[x, y]) for y in range(b.shape[1])] for x in range(b.shape[0])]
                t = time.time()
                R = exact.resultant_y(F, G)
                done[str(i)] = dict(record(R), seconds=round(time.time() - t, 2))
                print(f"O1 {name}[{i}]: {time.time() - t:.1f} s", flush=True)
                with open(o1_path, "w") as fh:
                    json.dump(o1, fh, indent=0, sort_keys=True)
                    fh.write("\n")


def _int(limbs):
    return int.from_bytes(np.ascontiguousarray(limbs, dtype="<u4").tobytes(), "little", signed=True)


if __name__ == "__main__":
    main()
