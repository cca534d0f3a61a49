"""Error of the FP32-storage path against the FP64 oracle for each
single-tensor configuration (the 8^6 correctness case, the 3D benchmark
tensor A[48^3,16^3], the 4D tensor A[12^8] and the differentiable A[10^8]),
written as a markdown table. Needs a GPU; run from the repository root:

    python -m tests.report_fp32_config_errors > profiles/fp32_error_per_config.md

A is generated in FP64, rounded to FP32 on the device and summed in FP32
storage and arithmetic; the oracle runs on the FP64 inputs. Columns as in
tests/report_fp32_errors.py: L = 1-norm of the operator, err = max |B_fp32 -
B_oracle|, rel = err / (L max|A|), bound (terms + 2) 2^-24."""
import math
import sys

import numpy as np


def main():
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    import workloads as wl
    from tests.gpu_helpers import chain_norm, nterms
    cases = [
        ("3D 8^6", wl.config1(), ["row1", "row2", "row3", "row4", "random"]),
        ("3D A[48^3,16^3]", wl.config2(), ["row1", "row2", "random"]),
        ("4D A[12^8]", wl.config3(), ["row5", "row6", "row18", "random"]),
        ("4D A[10^8]", wl.config5(), ["random", "row5"]),
    ]
    print("# FP32 storage per configuration: error against the FP64 oracle\n")
    print("Command: `python -m tests.report_fp32_config_errors` (FP32 storage and")
    print("arithmetic on the GPU, the oracle on the FP64 inputs).\n")
    print("| configuration | set | factorized | L | max abs A | err | rel = err/(L max abs A) | bound (terms+2) 2^-24 |")
    print("|---|---|---|---|---|---|---|---|")
    worst = 0.0
    for label, cfg, names in cases:
        shape = tuple(cfg.spec) + (cfg.O,) * cfg.d
        A_np = wl.uniform(cfg.seed, shape)
        A = ss.to_colmajor(torch.from_numpy(A_np).to("cuda").to(torch.float32))
        B = ss.colmajor_like(A)
        amax = float(np.abs(A_np).max())
        for name in names:
            coef = np.atleast_2d(cfg.sets[name])
            fac = coef.shape[0] > 1
            ss.spinsum(A, coef, d=cfg.d, out=B, factorized=fac)
            torch.cuda.synchronize()
            want = oracle.spinsum(A_np, cfg.d, coef, factorized=fac)
            got = B.double().cpu().numpy()
            err = float(np.abs(got - want).max())
            L = chain_norm(cfg.d, coef, fac)
            rel = err / (L * amax)
            bound = (nterms(cfg.d, coef, fac) + 2) * 2.0 ** -24
            worst = max(worst, rel / bound)
            print(f"| {label} | {name} | {'yes' if fac else 'no'} | {L:g} | {amax:.4f} | {err:.3e} | {rel:.3e} | "
                  f"{bound:.2e} |")
            del want, got
        del A, B, A_np
        torch.cuda.empty_cache()
    print(f"\nLargest rel / bound over all rows: {worst:.3f}.")
    return 0


if __name__ == "__main__":
    sys.exit(main())
