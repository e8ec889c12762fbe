"""Chain diagnostics on the GPU against the FP64 oracle (oracle/diagnostics.py).

Nested R-hat (Sec. 3.2; Margossian et al. 2024) to 1e-12 relative in both
height precisions, including one draw per chain (N = 1), one chain per
super-chain (M = 1) and identical super-chains (exactly 1); the tomographic
standard deviation of the below-interface indicators (Eq.
def_below_interface_indicator) bit for bit, with heights placed exactly on
voxel levels (eta(0) = 1/2), a ragged sample count and the scenario size.
"""
import numpy as np
import pytest
import torch

from oracle import diagnostics as D
from paper_2603_28907_gb300 import mt, workloads as W
from tests.gpu_common import DEV

pytestmark = pytest.mark.gpu


def _ctx(w, precision):
    return mt.from_workload(W.problem(w), precision=precision)


def _dtype(precision):
    return torch.float64 if precision == mt.PREC_F64 else torch.float32


@pytest.mark.parametrize("precision", [mt.PREC_F32, mt.PREC_F64])
@pytest.mark.parametrize("shape", [(3, 16, 4), (1, 24, 6), (5, 6, 6)])   # (N, C, n_super)
def test_nested_rhat_matches_oracle(precision, shape):
    N, C, K = shape
    w = W.tiny()
    ctx = _ctx(w, precision)
    rng = np.random.default_rng(11 + N + C)
    base = np.stack([W.init_chains(w, C)] * N)                       # [N][C][L][R][Q]
    noise = rng.standard_normal(base.shape) * 0.3
    shift = rng.standard_normal((1, K, 1, 1, 1, 1)) * 0.5            # per super-chain offsets
    d = base + noise + np.repeat(shift, C // K, axis=1).reshape(1, C, 1, 1, 1) * np.ones_like(base)
    dt = torch.tensor(d, dtype=_dtype(precision), device=DEV).contiguous()
    P = w.L * w.R * w.Q
    r = torch.zeros(P, dtype=torch.float64, device=DEV)
    rmax = ctx.nested_rhat(dt, K, r)
    ref = D.nested_rhat(dt.cpu().double().numpy().reshape(N, C, P), K)
    np.testing.assert_allclose(r.cpu().numpy(), ref, rtol=1e-12, atol=0)
    assert abs(rmax - ref.max()) <= 1e-12 * ref.max()
    ctx.close()


def test_nested_rhat_identical_super_chains_is_one():
    w = W.tiny()
    ctx = _ctx(w, mt.PREC_F32)
    one = np.stack([W.init_chains(w, 4)] * 2)                         # N=2, M=4
    d = np.concatenate([one, one, one], axis=1)                       # 3 super-chains alike
    dt = torch.tensor(d, dtype=torch.float32, device=DEV).contiguous()
    r = torch.zeros(w.L * w.R * w.Q, dtype=torch.float64, device=DEV)
    assert ctx.nested_rhat(dt, 3, r) == 1.0
    assert torch.all(r == 1.0)
    ctx.close()


def test_nested_rhat_rejects_bad_grouping():
    w = W.tiny()
    ctx = _ctx(w, mt.PREC_F32)
    dt = torch.zeros((1, 10, w.L, w.R, w.Q), dtype=torch.float32, device=DEV)
    with pytest.raises(mt.MtError):
        ctx.nested_rhat(dt, 3)                                        # 3 does not divide 10
    with pytest.raises(mt.MtError):
        ctx.nested_rhat(dt, 1)
    ctx.close()


@pytest.mark.parametrize("precision", [mt.PREC_F32, mt.PREC_F64])
def test_interface_std_bit_exact_with_ties(precision):
    w = W.tiny()                                                      # 3 surfaces, 16 x 16, Lz 150
    ctx = _ctx(w, precision)
    S, n_z = 37, 150                                                  # levels z_k = k (exact)
    H = W.init_chains(w, S)
    H[::3, 1, 2:9, 4] = 70.0                                          # on a level: eta(0) = 1/2
    H[1::5, 0, :, 7] = np.round(H[1::5, 0, :, 7])
    Ht = torch.tensor(H, dtype=_dtype(precision), device=DEV).contiguous()
    out = torch.zeros((w.L, n_z, w.R, w.Q), dtype=torch.float64, device=DEV)
    ctx.interface_std(Ht, n_z, out)
    ref = D.interface_std(Ht.cpu().double().numpy(), w.box[2], n_z)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert float(out.max()) <= 0.5
    ctx.close()


def test_interface_std_scenario_size():
    w = W.scenario()
    ctx = _ctx(w, mt.PREC_F32)
    S, n_z = 1024, 30
    H = W.init_chains(w, S)
    Ht = torch.tensor(H, dtype=torch.float32, device=DEV).contiguous()
    out = torch.zeros((w.L, n_z, w.R, w.Q), dtype=torch.float64, device=DEV)
    ctx.interface_std(Ht, n_z, out)
    ref = D.interface_std(Ht.cpu().double().numpy(), w.box[2], n_z)
    assert np.array_equal(out.cpu().numpy(), ref)
    with pytest.raises(mt.MtError):
        ctx.interface_std(Ht, 0, out)
    ctx.close()
