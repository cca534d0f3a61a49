"""d = 2 (the CCSD case: a 4-index tensor with the pair (i, j) permuted) and
the general symmetrizers / antisymmetrizers (coefficients 1 and sign(sigma))
for d = 2, 3, 4, through the C-ABI against the oracle: the orbit-stream
kernel (spectators), the tiled kernel (the N^2 matrix, ragged N), the
general-stride kernel, FP32 storage, in place, beta and a batched plan that
mixes d = 2 and d = 3 problems."""
import itertools

import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact, assert_within, fp32_tol, fp64_tol, gpu_run

pytestmark = pytest.mark.gpu

SETS2 = {"sym": [[1.0, 1.0]], "antisym": [[1.0, -1.0]], "ccsd": [[2.0, -1.0]], "chain": [[2.0, -1.0], [1.0, 3.0]]}


def _sign(p):
    s = 1
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if p[i] > p[j]:
                s = -s
    return s


@pytest.fixture(scope="module")
def orc():
    import oracle
    return oracle


@pytest.mark.parametrize("name", sorted(SETS2))
@pytest.mark.parametrize("shape", [(40, 40, 24, 24), (7, 5, 13, 13), (64, 64)], ids=["spectators", "small-spectators", "matrix"])
def test_d2_sets(orc, name, shape):
    coef = np.array(SETS2[name])
    fac = coef.shape[0] > 1
    A = wl.uniform(70, shape)
    want = orc.spinsum(A, 2, coef, factorized=fac)
    assert_within(gpu_run(A, 2, coef, factorized=fac), want, fp64_tol(2, coef, fac, A), name)
    assert_bitexact(gpu_run(A, 2, coef, factorized=fac, strict=True), want, name + " strict")
    Ai = wl.integers(71, shape)
    wi = orc.spinsum(Ai, 2, coef, factorized=fac)
    assert_bitexact(gpu_run(Ai, 2, coef, factorized=fac), wi, name + " integer")
    assert_bitexact(gpu_run(Ai, 2, coef, factorized=fac, inplace=True), wi, name + " integer in place")
    Af = A.astype(np.float32).astype(np.float64)
    assert_within(gpu_run(Af, 2, coef, factorized=fac, dtype="f32"), orc.spinsum(Af, 2, coef, factorized=fac),
                  fp32_tol(2, coef, fac, Af), name + " fp32")


@pytest.mark.parametrize("N", [33, 70, 130])
def test_d2_paper_layout_ragged(orc, N):
    """N x N matrices whose edge is not a multiple of the 32 x 32 tile."""
    coef = np.array([[2.0, -1.0]])
    A = wl.uniform(72, (N, N))
    B0 = wl.uniform(73, (N, N))
    want = 0.5 * orc.spinsum(A, 2, coef) - 1.5 * B0
    assert_within(gpu_run(A, 2, coef, alpha=0.5, beta=-1.5, B0=B0), want, 4 * fp64_tol(2, coef, False, A), "beta")
    Ai = wl.integers(74, (N, N))
    assert_bitexact(gpu_run(Ai, 2, coef, inplace=True), orc.spinsum(Ai, 2, coef), "in place")
    assert_bitexact(gpu_run(Ai, 2, coef, offset=1), orc.spinsum(Ai, 2, coef), "misaligned")


def test_d2_general_strides(orc):
    coef = np.array([[1.0, -1.0]])
    A = wl.uniform(75, (6, 5, 9, 9))
    want = orc.spinsum(A, 2, coef)
    for layout in ("rowmajor", "sliced"):
        assert_bitexact(gpu_run(A, 2, coef, layout=layout, strict=True), want, layout)
        assert_within(gpu_run(A, 2, coef, layout=layout), want, fp64_tol(2, coef, False, A), layout)


@pytest.mark.parametrize("d,shape", [(2, (16, 16, 20, 20)), (3, (8, 8, 8, 9, 9, 9)), (4, (3, 3, 3, 3, 6, 6, 6, 6))])
@pytest.mark.parametrize("kind", ["symmetrizer", "antisymmetrizer"])
def test_symmetrizers(orc, d, shape, kind):
    """sum_sigma pi_sigma (A) is symmetric and sum_sigma sign(sigma) pi_sigma (A)
    antisymmetric under every transposition of the permuted indices; both
    equal the oracle bit for bit on integer-valued inputs."""
    perms = list(itertools.permutations(range(d)))
    coef = np.array([[1.0 if kind == "symmetrizer" else float(_sign(p)) for p in perms]])
    Ai = wl.integers(76 + d, shape)
    got = gpu_run(Ai, d, coef)
    assert_bitexact(got, orc.spinsum(Ai, d, coef), kind)
    s = 1.0 if kind == "symmetrizer" else -1.0
    for a, b in itertools.combinations(range(d), 2):
        axes = list(range(2 * d))
        axes[d + a], axes[d + b] = axes[d + b], axes[d + a]
        assert np.array_equal(got.transpose(axes), s * got), (kind, a, b)


def test_batched_plan_mixes_d2_and_d3(orc):
    import torch
    import paper_1705_06661_gb300 as ss
    probs = [(2, (30, 30, 16, 16), np.array([[2.0, -1.0]])), (3, (9, 9, 9, 7, 7, 7), wl.table2(1)),
             (2, (7, 9, 11, 11), np.array([[1.0, 1.0]])), (2, (100, 100), np.array([[1.0, -1.0]]))]
    specs, keep = [], []
    for i, (d, shp, coef) in enumerate(probs):
        A_np = wl.uniform(80 + i, shp)
        a = ss.to_colmajor(torch.from_numpy(A_np).cuda())
        b = ss.colmajor_like(a)
        specs.append({"A": a, "B": b, "coef": coef, "d": d, "factorized": coef.shape[0] > 1})
        keep.append((d, A_np, coef, b))
    plan = ss.Plan(specs, tune=False)
    plan.execute()
    torch.cuda.synchronize()
    for d, A_np, coef, b in keep:
        want = orc.spinsum(A_np, d, coef, factorized=coef.shape[0] > 1)
        assert_within(b.cpu().numpy(), want, fp64_tol(d, coef, coef.shape[0] > 1, A_np), f"batched d={d}")
    plan.close()
