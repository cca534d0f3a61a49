"""Error of the FP32-storage path against the FP64 oracle, per block of the
batched workload (64 uneven 3D blocks, one persistent launch), written as a
markdown table. Needs a GPU; run from the repository root:

    python -m tests.report_fp32_errors > profiles/fp32_error_batched_64_blocks.md

Columns: L = 1-norm of the operator (factor norms multiplied for a chain),
err = max |B_fp32 - B_oracle| over the block with the oracle on the FP64
inputs, rel = err / (L * max|A|), and the stated bound
(terms + 2) * 2^-24 * L * max|A| relative, i.e. (terms + 2) * 2^-24."""
import math
import sys

import numpy as np


def main():
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    import workloads as wl
    from tests.gpu_helpers import chain_norm
    blocks = wl.config4_blocks()
    devA, devB, specs, host = [], [], [], []
    for pr in blocks:
        A_np = wl.uniform(pr.seed, pr.shape)
        a = torch.from_numpy(A_np).to("cuda").to(torch.float32)
        a = ss.to_colmajor(a)
        b = ss.colmajor_like(a)
        devA.append(a)
        devB.append(b)
        host.append(A_np)
        specs.append({"A": a, "B": b, "coef": pr.coef, "d": 3, "factorized": True})
    plan = ss.Plan(specs, tune=False)
    plan.execute()
    torch.cuda.synchronize()
    print("# FP32 storage, batched 64 uneven 3D blocks: error against the FP64 oracle\n")
    print("Command: `python -m tests.report_fp32_errors` (one persistent FP32 launch of the")
    print("batched plan; the oracle runs on the FP64 inputs).\n")
    print("| block | shape | set | L | max abs A | err | rel = err/(L max abs A) | bound (terms+2) 2^-24 |")
    print("|---|---|---|---|---|---|---|---|")
    worst = 0.0
    for pr, A_np, b in zip(blocks, host, devB):
        want = oracle.spinsum(A_np, 3, pr.coef, factorized=True)
        got = b.double().cpu().numpy()
        err = float(np.abs(got - want).max())
        L = chain_norm(3, pr.coef, True)
        amax = float(np.abs(A_np).max())
        rel = err / (L * amax)
        c = np.atleast_2d(pr.coef)
        terms = int(sum(np.count_nonzero(f) for f in c))
        bound = (terms + 2) * 2.0 ** -24
        worst = max(worst, rel)
        print(f"| {pr.name} | V={pr.spec[0]}, O={pr.O} | {c.shape[0]} factor(s), {terms} terms | {L:g} | {amax:.4f} | "
              f"{err:.3e} | {rel:.3e} | {bound:.2e} |")
    plan.close()
    print(f"\nWorst relative error over the 64 blocks: {worst:.3e} "
          f"(2^{math.log2(worst):.1f}); FP64 storage on the same plan is within 1e-14 relative.")
    return 0


if __name__ == "__main__":
    sys.exit(main())
