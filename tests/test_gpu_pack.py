"""Packed antisymmetric storage on the GPU (spinsum_unpack / spinsum_pack)
against the oracle's definitions: d = 2, 3, 4, FP64 and FP32, 16-byte and
misaligned runs, the paper's layout (no spectators), and the round trip."""
import math

import numpy as np
import pytest

import workloads as wl
from tests.gpu_helpers import assert_bitexact

pytestmark = pytest.mark.gpu

CASES = [(2, (6, 10), 9), (2, (5, 3), 17), (3, (4, 6, 8), 7), (3, (1, 1, 1), 9), (4, (3, 4, 2, 2), 6),
         (4, (2, 3, 5, 1), 7)]


def _colmajor(x, dtype, offset=0):
    import torch
    import paper_1705_06661_gb300 as ss
    if offset == 0:
        return ss.to_colmajor(torch.from_numpy(x).to(dtype).cuda())
    n = x.size
    base = torch.zeros(n + offset, dtype=dtype, device="cuda")
    t = base[offset:].view(tuple(reversed(x.shape))).permute(*reversed(range(x.ndim)))
    t.copy_(torch.from_numpy(x).to(dtype).cuda())
    return t


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("d,spec,O", CASES)
def test_unpack_pack_match_oracle(d, spec, O, dt, offset):
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    tdt = torch.float64 if dt == "f64" else torch.float32
    P_np = wl.uniform(95 + d, tuple(spec) + (math.comb(O, d),))
    if dt == "f32":
        P_np = P_np.astype(np.float32).astype(np.float64)
    want = oracle.unpack(P_np, d, O)
    P = _colmajor(P_np, tdt, offset)
    B = ss.colmajor_empty(tuple(spec) + (O,) * d, dtype=tdt)
    B.fill_(float("nan"))                  # every element must be written
    ss.unpack(P, d, O, out=B)
    torch.cuda.synchronize()
    assert_bitexact(B.double().cpu().numpy(), want, f"unpack d={d}")
    B2 = _colmajor(want, tdt, offset)
    P2 = ss.pack(B2, d)
    torch.cuda.synchronize()
    assert_bitexact(P2.double().cpu().numpy(), P_np, f"pack d={d}")


def test_paper_layout_round_trip():
    """no spectators: the O^3 tensor and its C(O, 3) packed values"""
    import torch
    import oracle
    import paper_1705_06661_gb300 as ss
    O = 40
    P_np = wl.uniform(99, (1, 1, 1, math.comb(O, 3)))
    P = _colmajor(P_np, torch.float64)
    B = ss.unpack(P, 3, O)
    torch.cuda.synchronize()
    Bn = B.cpu().numpy()
    assert_bitexact(Bn, oracle.unpack(P_np, 3, O), "unpack")
    assert_bitexact(ss.pack(B, 3).cpu().numpy(), P_np, "pack")


def test_pack_argument_errors():
    import torch
    import paper_1705_06661_gb300 as ss
    P = ss.colmajor_empty((2, 2, 2, math.comb(5, 3)))
    with pytest.raises(ValueError):
        ss.unpack(P, 3, 6)                 # packed extent does not match O
    B = ss.colmajor_empty((2, 2, 2, 5, 5, 5))
    with pytest.raises(ss.SpinsumError):
        ss.unpack(P, 3, 5, out=B[:, :, :, :, :, :].transpose(0, 1))  # spectators not dense and fastest
    overlap = torch.empty(4096, dtype=torch.float64, device="cuda")
    Pv = overlap[:2 * 2 * 2 * 10].view(10, 2, 2, 2).permute(3, 2, 1, 0)
    Bv = overlap[:1000].view(5, 5, 5, 2, 2, 2).permute(5, 4, 3, 2, 1, 0)
    with pytest.raises(ss.SpinsumError):
        ss.unpack(Pv, 3, 5, out=Bv)
