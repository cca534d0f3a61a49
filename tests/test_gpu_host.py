"""Host-resident tensors (spinsum_2d_host / spinsum_3d_host / spinsum_4d_host): chunked,
pipelined copy-in / sum / copy-out against the oracle, with pinned and
pageable memory, in place, with beta, and with a workspace of one slice."""
import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact, assert_within, fp64_tol

pytestmark = pytest.mark.gpu


def _cpu(A_np, pinned):
    import torch
    import paper_1705_06661_gb300 as ss
    t = ss.colmajor_empty(A_np.shape, device="cpu")
    if pinned:
        t = torch.empty(tuple(reversed(A_np.shape)), dtype=torch.float64).pin_memory().permute(
            *reversed(range(A_np.ndim)))
    t.copy_(torch.from_numpy(A_np))
    return t


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("d,shape", [(2, (9, 7, 11, 11)), (3, (6, 5, 9, 5, 5, 5)), (4, (3, 4, 2, 5, 4, 4, 4, 4))])
def test_host_pipeline_matches_oracle(d, shape, pinned):
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    coef = {2: np.array([[2.0, -1.0]]), 3: wl.table2(1), 4: wl.table2(5)}[d]
    for kind in ("int", "uni"):
        A_np = (wl.integers if kind == "int" else wl.uniform)(31, shape)
        want = oracle.spinsum(A_np, d, coef, factorized=True)
        A = _cpu(A_np, pinned)
        out = ss.spinsum_host(A, coef, d=d, factorized=True)
        torch.cuda.synchronize()
        if kind == "int":
            assert_bitexact(out.numpy(), want, "host pipeline")
        else:
            assert_within(out.numpy(), want, fp64_tol(d, coef, True, A_np), "host pipeline")


@pytest.mark.parametrize("pinned", [False, True])
def test_host_pipeline_inplace_beta_and_small_workspace(pinned):
    """pageable memory: the staged pipeline in a workspace of one slice;
    pinned memory: the zero-copy kernel (the workspace is not used)."""
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    shape = (4, 4, 7, 6, 6, 6)
    coef = wl.random_coef(3, 33)
    A_np = wl.integers(34, shape)
    B_np = wl.integers(35, shape)
    # one slice of workspace (7 chunks of the slowest spectator index)
    one_slice = 4 * 4 * 6 ** 3 * 8
    ws = torch.empty(3 * one_slice, dtype=torch.uint8, device="cuda")
    A = _cpu(A_np, pinned)
    ss.spinsum_host(A, coef, inplace=True, workspace=ws)
    torch.cuda.synchronize()
    assert_bitexact(A.numpy(), oracle.spinsum(A_np, 3, coef), "in place")
    A = _cpu(A_np, pinned)
    B = _cpu(B_np, pinned)
    ws2 = torch.empty(6 * one_slice, dtype=torch.uint8, device="cuda")
    ss.spinsum_host(A, coef, out=B, alpha=-2.0, beta=3.0, workspace=ws2)
    torch.cuda.synchronize()
    want = oracle.spinsum(A_np, 3, coef, alpha=-2.0, beta=3.0, B=np.asfortranarray(B_np.copy()))
    assert_bitexact(B.numpy(), want, "beta")
    if not pinned:
        with pytest.raises(ss.SpinsumError, match="workspace too small"):
            ss.spinsum_host(A, coef, out=B, workspace=torch.empty(100, dtype=torch.uint8, device="cuda"))
