"""Tensor-core rate of the library's own distance GEMM, per operand precision.

Times the GEMM kernel of gbk_pairwise_distances (inner products, every output written;
the kernel's own CUDA-event time from the library's profiler, not the operand
preparation) at a shape where the tensor cores, not the output stores, bound it:
nq = 8,192 queries against nb = 16,384 rows of d = 8,192 (2 d flops per 4 output bytes).  The
default float32-accurate precision issues three FP16 MMAs per product (hi x hi, hi x lo,
lo x hi; reported as "fp16"), the TF32 split three TF32 MMAs (reported as "tf32"): their
executed rates are three times their algorithmic rates.  The kernel's own CUDA-event time
on the launching stream, one warm-up and `reps` timed calls.  The result is a rate this
kernel reaches, i.e. a lower bound of the hardware's.

    python -m paper_1702_08734_gb300.peaks [out.json]
"""
from __future__ import annotations

import json
import sys
import time


def measure(reps: int = 3, nq: int = 8192, nb: int = 16384, d: int = 8192):
    import torch

    import paper_1702_08734_gb300 as g
    from paper_1702_08734_gb300 import datagen
    g.load()
    xq = datagen.gaussian_matrix_cuda(11, nq, d)
    xb = datagen.gaussian_matrix_cuda(12, nb, d)
    flops = 2.0 * nq * nb * d
    out = {"shape": {"nq": nq, "nb": nb, "d": d}, "reps": reps,
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "gpu": torch.cuda.get_device_name(0)}
    kern = {"fp32": "dist_gemm_fp16x3", "tf32x3": "dist_gemm_tf32x3", "bf16": "dist_gemm_bf16",
            "fp8": "dist_gemm_fp8"}
    names = {"fp32": "fp16", "tf32x3": "tf32", "bf16": "bf16", "fp8": "fp8"}
    for prec, passes in (("tf32x3", 3), ("fp32", 3), ("bf16", 1), ("fp8", 1)):
        g.pairwise_distances(xq, xb, metric="ip", precision=prec)
        torch.cuda.synchronize()
        g.profile_enable(True)
        for _ in range(reps):
            g.pairwise_distances(xq, xb, metric="ip", precision=prec)
        torch.cuda.synchronize()
        g.profile_enable(False)
        times = [t for nm, t in g.profile_read() if nm == kern[prec]]
        ms = sum(times) / len(times)
        name = names[prec]
        out[name + "_tflops"] = passes * flops / (ms / 1e3) / 1e12
        out[name + "_ms"] = ms
    out["note"] = ("executed tensor-core rate of the library's pairwise GEMM kernel (its output "
                   "stores included, operand preparation not); tf32 and fp16 count the 3 MMAs of "
                   "the float32-accurate splits")
    return out


if __name__ == "__main__":
    res = measure()
    js = json.dumps(res, indent=1)
    if len(sys.argv) > 1:
        with open(sys.argv[1], "w") as f:
            f.write(js + "\n")
    print(js)
