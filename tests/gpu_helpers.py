"""Shared helpers of the GPU tests: run the CUDA path through the C-ABI binding
on numpy inputs and state the tolerances."""
import math

import numpy as np


def ss():
    import paper_1705_06661_gb300 as m
    return m


def chain_norm(d, coef, factorized):
    """L of the tolerance 1e-14 * L * max|A|: |alpha|_1 of the expanded
    operator, or the product of the factor 1-norms for a factorized chain."""
    import oracle
    c = np.atleast_2d(np.asarray(coef, dtype=np.float64))
    if factorized and c.shape[0] > 1:
        return float(np.prod([np.abs(f).sum() for f in c]))
    return float(np.abs(oracle.expand(d, c)).sum())


def fp64_tol(d, coef, factorized, A, alpha=1.0):
    return 1e-14 * chain_norm(d, coef, factorized) * max(float(np.abs(A).max()), 1e-300) * abs(alpha)


def gpu_run(A_np, d, coef, *, factorized=False, strict=False, adjoint=False, alpha=1.0, beta=0.0, inplace=False,
            B0=None, dtype="f64", layout="colmajor", offset=0, tma=False):
    """Copy A (numpy, any strides) to the GPU in the requested layout, run the
    spin summation through the C-ABI, return the result as numpy float64."""
    import torch
    m = ss()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dev = torch.device("cuda:0")

    def place(x):
        t = torch.from_numpy(np.ascontiguousarray(x.astype(np.float64 if dtype == "f64" else np.float32)))
        if layout == "colmajor":
            if offset:
                n = x.size + offset
                base = torch.empty(n, dtype=tdt, device=dev)
                g = base[offset:].view(tuple(reversed(x.shape))).permute(*reversed(range(x.ndim)))
                g.copy_(t.to(dev))
                return g
            return m.to_colmajor(t.to(dev))
        if layout == "rowmajor":
            return t.to(dev).contiguous()
        if layout == "sliced":   # non-dense spectator strides
            big = m.colmajor_empty((x.shape[0] + 2,) + x.shape[1:], dtype=tdt, device=dev)
            g = big[1:1 + x.shape[0]]
            g.copy_(t.to(dev))
            return g
        raise ValueError(layout)

    A = place(A_np)
    if inplace:
        out = A
    elif B0 is not None:
        out = place(B0)
    else:
        out = m.colmajor_like(A) if layout != "rowmajor" else torch.empty_like(A)
    m.spinsum(A, coef, d=d, out=None if inplace else out, factorized=factorized, strict=strict, adjoint=adjoint,
              alpha=alpha, beta=beta, inplace=inplace, tma=tma)
    m.spinsum_check_status(torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy().astype(np.float64)


def assert_bitexact(got, want, msg=""):
    if not np.array_equal(got, want, equal_nan=True):
        bad = np.argwhere(~((got == want) | (np.isnan(got) & np.isnan(want))))
        i = tuple(bad[0])
        raise AssertionError(f"{msg}: {len(bad)} mismatches, first at {i}: got {got[i]!r} want {want[i]!r}")


def assert_within(got, want, tol, msg=""):
    err = float(np.max(np.abs(got - want))) if got.size else 0.0
    if not err <= tol:
        raise AssertionError(f"{msg}: max |dB| = {err:.3e} > tol {tol:.3e}")
    return err


def nterms(d, coef, factorized):
    import oracle
    c = np.atleast_2d(np.asarray(coef, dtype=np.float64))
    if factorized and c.shape[0] > 1:
        return int(sum(np.count_nonzero(f) for f in c))
    return int(np.count_nonzero(oracle.expand(d, c)))


def fp32_tol(d, coef, factorized, A):
    """FP32 storage and accumulation: every input rounding, product and sum
    contributes at most 2^-24 relative to L max|A|; the bound adds one unit
    per term and two for the input and output roundings."""
    return (nterms(d, coef, factorized) + 2) * 2.0 ** -24 * chain_norm(d, coef, factorized) * float(np.abs(A).max())


def fact(d):
    return math.factorial(d)
