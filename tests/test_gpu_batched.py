"""Batched plans: many uneven 3D blocks (the shape mix of the batched
workload, scaled down so the oracle finishes in seconds) in one persistent
launch; parity per block with the oracle, FP32 storage error per block, CUDA
graph capture and replay, autotuned and heuristic tilings."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact, assert_within, fp32_tol, fp64_tol

pytestmark = pytest.mark.gpu


def small_blocks(n=64, seed=3):
    """Same recipe as the batched workload (V = lo + r mod span, O likewise,
    coefficient sets cycling Table II rows 1-4 and a random set) with
    V in [3, 14] and O in [2, 9]."""
    x = wl.draws(seed, 2 * n) >> np.uint64(32)
    out = []
    for b in range(n):
        V = 3 + int(x[2 * b] % np.uint64(12))
        O = 2 + int(x[2 * b + 1] % np.uint64(8))
        k = b % 5
        coef = wl.table2(k + 1) if k < 4 else wl.random_coef(3, 200 + b)
        out.append(wl.Problem(3, (V, V, V), O, 1000 + b, coef, f"block{b}"))
    return out


def _run(problems, kind, dtype, inplace, tune, factorized=True, graph=False):
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    tdt = torch.float64 if dtype == "f64" else torch.float32
    host, devA, devB, specs = [], [], [], []
    for pr in problems:
        A = (wl.integers if kind == "int" else wl.uniform)(pr.seed, pr.shape)
        if dtype == "f32":
            A = np.asfortranarray(A.astype(np.float32).astype(np.float64))
        host.append(A)
        a = ss.to_colmajor(torch.from_numpy(A).to("cuda", tdt))
        b = None if inplace else ss.colmajor_like(a)
        devA.append(a)
        devB.append(b)
        specs.append({"A": a, "B": b, "coef": pr.coef, "d": 3, "factorized": factorized})
    plan = ss.Plan(specs, tune=tune)
    if tune and inplace:
        # tuning runs executed the in-place problems: restore the inputs
        for a, A in zip(devA, host):
            a.copy_(torch.from_numpy(A).to("cuda", tdt))
    if graph:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                plan.execute()
        torch.cuda.current_stream().wait_stream(s)
        g.replay()
    else:
        plan.execute()
    torch.cuda.synchronize()
    ss.spinsum_check_status(torch.cuda.current_stream().cuda_stream)
    desc = plan.describe()
    results = [(a if b is None else b).double().cpu().numpy() for a, b in zip(devA, devB)]
    wants = [oracle.spinsum(A, 3, pr.coef, factorized=factorized) for A, pr in zip(host, problems)]
    plan.close()
    return host, results, wants, desc


@pytest.mark.parametrize("inplace", [False, True])
@pytest.mark.parametrize("tune", [False, True])
def test_batched_fp64(inplace, tune):
    probs = small_blocks()
    for kind in ("int", "uni"):
        host, got, want, desc = _run(probs, kind, "f64", inplace, tune)
        assert "classes=1" in desc and "problems=64" in desc, desc
        for pr, A, g, w in zip(probs, host, got, want):
            if kind == "int":
                assert_bitexact(g, w, pr.name)
            else:
                assert_within(g, w, fp64_tol(3, pr.coef, True, A), pr.name)


def test_batched_graph_replay():
    probs = small_blocks(40, seed=5)
    host, got, want, _ = _run(probs, "int", "f64", False, True, graph=True)
    for pr, g, w in zip(probs, got, want):
        assert_bitexact(g, w, pr.name)


def test_batched_fp32_error_per_block():
    probs = small_blocks(64, seed=6)
    host, got, want, _ = _run(probs, "uni", "f32", False, False)
    worst = 0.0
    for pr, A, g, w in zip(probs, host, got, want):
        tol = fp32_tol(3, pr.coef, True, A)
        err = assert_within(g, w, tol, pr.name)
        L = np.prod([np.abs(f).sum() for f in np.atleast_2d(pr.coef)])
        worst = max(worst, err / (L * np.abs(A).max()))
    assert worst < 2.0 ** -19


def test_mixed_dimensions_and_layouts():
    """d = 3 and d = 4 problems, a row-major (general kernel) problem and an
    empty one in one plan."""
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    A3 = wl.integers(1, (5, 6, 7, 4, 4, 4))
    A4 = wl.integers(2, (3, 3, 3, 3, 5, 5, 5, 5))
    Ar = wl.integers(3, (4, 4, 4, 5, 5, 5))
    a3 = ss.to_colmajor(torch.from_numpy(A3).cuda())
    a4 = ss.to_colmajor(torch.from_numpy(A4).cuda())
    ar = torch.from_numpy(np.ascontiguousarray(Ar)).cuda()
    ae = ss.colmajor_empty((0, 3, 3, 4, 4, 4))
    b3, b4, br, be = ss.colmajor_like(a3), ss.colmajor_like(a4), torch.empty_like(ar), ss.colmajor_like(ae)
    plan = ss.Plan([{"A": a3, "B": b3, "coef": wl.table2(1), "d": 3},
                    {"A": a4, "B": b4, "coef": wl.table2(5), "d": 4, "factorized": True},
                    {"A": ar, "B": br, "coef": wl.random_coef(3, 9), "d": 3},
                    {"A": ae, "B": be, "coef": wl.table2(2), "d": 3}], tune=False)
    plan.execute()
    torch.cuda.synchronize()
    assert "general=1" in plan.describe()
    assert_bitexact(b3.cpu().numpy(), oracle.spinsum(A3, 3, wl.table2(1)), "3d")
    assert_bitexact(b4.cpu().numpy(), oracle.spinsum(A4, 4, wl.table2(5), factorized=True), "4d")
    assert_bitexact(br.cpu().numpy(), oracle.spinsum(Ar, 3, wl.random_coef(3, 9)), "row-major")
    plan.close()
