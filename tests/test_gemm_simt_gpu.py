"""GPU parity of the FP32 FFMA GEMM (64 x 64 tiles) against the FP64 oracle,
and its tile->program coverage against the oracle's enumeration."""
import numpy as np
import pytest
import torch

import paper_2606_15991_gb300 as tp
import synth
from oracle import gemm as ogemm
from oracle import partition as opart

pytestmark = pytest.mark.gpu


def _gemm(ctx, a, b, kind=tp.MAP_IDENTITY, P=0, group_m=1, count=False, bk=16, split_k=0):
    M, N = a.shape[0], b.shape[1]
    c = torch.full((M, N), float("nan"), device="cuda")
    p = tp.tp_partition_create(ctx, c, (64, 64))
    if kind != tp.MAP_IDENTITY:
        tp.tp_partition_map(p, kind, P)
    counts = owner = None
    if count:
        counts = torch.zeros(M * N, dtype=torch.int32, device="cuda")
        owner = torch.full((M * N,), -1, dtype=torch.int32, device="cuda")
    tp.tp_gemm(ctx, p, a, b, tp.gemm_config(group_m=group_m, bk=bk, split_k=split_k),
               tp.make_exec(write_counts=counts, write_owner=owner))
    tp.tp_partition_destroy(p)
    return c, counts, owner


def test_512_cubed_uniform_within_tolerance(ctx):
    """The 512^3 configuration: A, B ~ U[-1,1] from seed 0, 64 programs."""
    a = torch.from_numpy(synth.uniform(512 * 512, seed=0)).reshape(512, 512).cuda()
    b = torch.from_numpy(synth.uniform(512 * 512, seed=1)).reshape(512, 512).cuda()
    c, counts, owner = _gemm(ctx, a, b, count=True)
    err = ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), b.cpu()))
    assert err <= 1e-5
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), opart.gemm_owner_map(512, 512, 64, 64))
    assert int(owner.max()) == 63


@pytest.mark.parametrize("bk", [8, 16, 32])
def test_integer_inputs_bit_exact(ctx, bk):
    a = torch.from_numpy(synth.integers(512 * 512, seed=3, lo=-4, hi=4)).reshape(512, 512).cuda()
    b = torch.from_numpy(synth.integers(512 * 512, seed=4, lo=-4, hi=4)).reshape(512, 512).cuda()
    c, _, _ = _gemm(ctx, a, b, bk=bk)
    assert np.array_equal(c.cpu().double().numpy(), ogemm.gemm(a.cpu(), b.cpu()))


def test_identity_and_permutation_bit_exact(ctx):
    b = torch.from_numpy(synth.uniform(256 * 192, seed=5)).reshape(256, 192).cuda()
    c, _, _ = _gemm(ctx, torch.eye(256, device="cuda"), b)
    assert torch.equal(c, b)
    perm = torch.tensor([(37 * i + 11) % 256 for i in range(256)])
    P = torch.zeros(256, 256)
    P[torch.arange(256), perm] = 1.0
    c, _, _ = _gemm(ctx, P.cuda(), b)
    assert torch.equal(c, b[perm.cuda()])


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (17, 13, 11), (65, 129, 31), (100, 1, 300), (3, 200, 64),
                                   (129, 65, 0)])
def test_ragged_shapes(ctx, m, n, k):
    a = torch.from_numpy(synth.uniform(m * k, seed=m)).reshape(m, k).cuda()
    b = torch.from_numpy(synth.uniform(k * n, seed=n + 7)).reshape(k, n).cuda()
    c, counts, owner = _gemm(ctx, a, b, count=True)
    ref = ogemm.gemm(a.cpu(), b.cpu())
    assert np.max(np.abs(c.cpu().double().numpy() - ref)) <= 1e-6 * max(1, k)
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), opart.gemm_owner_map(m, n, 64, 64))


@pytest.mark.parametrize("P,group_m", [(5, 2), (1, 1), (25, 4), (7, 3)])
def test_mapped_strided_partition(ctx, P, group_m):
    m, n, k = 300, 260, 70
    a = torch.from_numpy(synth.uniform(m * k, seed=9)).reshape(m, k).cuda()
    b = torch.from_numpy(synth.uniform(k * n, seed=10)).reshape(k, n).cuda()
    c, counts, owner = _gemm(ctx, a, b, tp.MAP_STRIDED, P, group_m, count=True)
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), b.cpu())) <= 1e-5
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(),
                          opart.gemm_owner_map(m, n, 64, 64, P, "strided", group_m))


def test_queue_partition_and_transposed_operand(ctx):
    m, n, k = 200, 333, 129
    a = torch.from_numpy(synth.uniform(m * k, seed=11)).reshape(m, k).cuda()
    bt = torch.from_numpy(synth.uniform(k * n, seed=12)).reshape(n, k).cuda()
    b = bt.t()                                   # K x N view with strides (1, K)
    c, counts, owner = _gemm(ctx, a, b, tp.MAP_QUEUE, 6, 2, count=True)
    assert ogemm.rel_frobenius(c.cpu(), ogemm.gemm(a.cpu(), b.cpu())) <= 1e-5
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    o = owner.cpu().numpy()
    assert o.min() >= 0 and o.max() < 6


def test_gemm_shape_errors(ctx):
    a = torch.zeros(64, 32, device="cuda")
    b = torch.zeros(31, 64, device="cuda")
    c = torch.zeros(64, 64, device="cuda")
    p = tp.tp_partition_create(ctx, c, (64, 64))
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm(ctx, p, a, b)
    assert e.value.status == tp._lib.ERR_SHAPE
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm(ctx, p, c, c)                 # A aliases the output
    assert e.value.status == tp._lib.ERR_ALIAS
    tp.tp_partition_destroy(p)
    p = tp.tp_partition_create(ctx, c, (32, 32))
    with pytest.raises(tp.TPError) as e:
        tp.tp_gemm(ctx, p, torch.zeros(64, 64, device="cuda"), torch.zeros(64, 64, device="cuda"))
    assert e.value.status == tp._lib.ERR_UNSUPPORTED
    tp.tp_partition_destroy(p)


@pytest.mark.parametrize("S", [2, 4])
@pytest.mark.parametrize("bk", [8, 32])
def test_split_k_programs(ctx, S, bk):
    """split_k = S: each 64 x 64 tile program is a cluster of S CTAs that run
    contiguous K slices; CTA r adds the S partials of rows [r*64/S, +64/S)
    in slice order and stores them. Integer inputs are exact in FP32 in any
    order; U[-1,1] inputs stay within 1e-5; every element is stored once, by
    the program that owns its tile; two runs are bit-identical."""
    a = torch.from_numpy(synth.integers(512 * 512, seed=13, lo=-4, hi=4)).reshape(512, 512).cuda()
    b = torch.from_numpy(synth.integers(512 * 512, seed=14, lo=-4, hi=4)).reshape(512, 512).cuda()
    c, counts, owner = _gemm(ctx, a, b, bk=bk, split_k=S, count=True)
    assert np.array_equal(c.cpu().double().numpy(), ogemm.gemm(a.cpu(), b.cpu()))
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), opart.gemm_owner_map(512, 512, 64, 64))
    a = torch.from_numpy(synth.uniform(300 * 700, seed=15)).reshape(300, 700).cuda()
    b = torch.from_numpy(synth.uniform(700 * 260, seed=16)).reshape(700, 260).cuda()
    c1, _, _ = _gemm(ctx, a, b, bk=bk, split_k=S)
    c2, counts, owner = _gemm(ctx, a, b, tp.MAP_STRIDED, 7, 2, bk=bk, split_k=S, count=True)
    assert torch.equal(c1, c2)
    assert ogemm.rel_frobenius(c1.cpu(), ogemm.gemm(a.cpu(), b.cpu())) <= 1e-5
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    assert np.array_equal(owner.cpu().numpy(), opart.gemm_owner_map(300, 260, 64, 64, 7, "strided", 2))


def test_split_k_validation(ctx):
    a = torch.ones(128, 64, device="cuda")
    b = torch.ones(64, 128, device="cuda")
    with pytest.raises(tp.TPError) as e:
        _gemm(ctx, a, b, split_k=3)
    assert e.value.status == tp._lib.ERR_INVALID
    with pytest.raises(tp.TPError) as e:
        _gemm(ctx, a, b, split_k=8)
    assert e.value.status == tp._lib.ERR_INVALID
    with pytest.raises(tp.TPError) as e:
        _gemm(ctx, a, b, tp.MAP_QUEUE, 2, split_k=2)
    assert e.value.status == tp._lib.ERR_UNSUPPORTED
    c, _, _ = _gemm(ctx, a[:, :1], b[:1], split_k=4)     # one K slice: three CTAs add zero partials
    assert torch.equal(c, torch.ones(128, 128, device="cuda"))


@pytest.mark.parametrize("m,n,k,split,kind,P,group_m", [
    (512, 512, 512, 2, tp.MAP_IDENTITY, 0, 1),   # the benchmark configuration
    (512, 512, 512, 4, tp.MAP_IDENTITY, 0, 1),
    (65, 132, 36, 1, tp.MAP_IDENTITY, 0, 1),     # ragged tiles, a partial K chunk
    (100, 4, 300, 1, tp.MAP_IDENTITY, 0, 1),
    (300, 200, 1000, 1, tp.MAP_STRIDED, 5, 1),   # programs walking several tiles
    (450, 260, 520, 1, tp.MAP_STRIDED, 7, 3),    # ... in raster bands of 3 tile rows
    (200, 300, 4104, 2, tp.MAP_STRIDED, 20, 2),  # split programs, one tile each, long K
])
def test_tma_fed_kernel_equals_register_staged(ctx, m, n, k, split, kind, P, group_m):
    """With 32-wide K steps, unit-stride 16-byte-aligned operands and an
    identity or strided map, the FP32 GEMM runs the TMA-fed kernel; the same
    values with A 4 bytes off alignment run the register-staged kernel. Both
    take each output's K sum in the same order (and split-K slices in slice
    order), so C is equal bit for bit; C is within 1e-5 of the FP64 oracle and
    every element is written once by the oracle's owner."""
    a = torch.from_numpy(synth.uniform(m * k, seed=m + k)).reshape(m, k).cuda()
    b = torch.from_numpy(synth.uniform(k * n, seed=n + 7)).reshape(k, n).cuda()
    c_tma, counts, owner = _gemm(ctx, a, b, kind, P, group_m=group_m, bk=32, split_k=split, count=True)
    abuf = torch.empty(m * k + 1, device="cuda")
    a_off = abuf[1:].view(m, k)
    a_off.copy_(a)
    c_reg, _, _ = _gemm(ctx, a_off, b, kind, P, group_m=group_m, bk=32, split_k=split)
    assert torch.equal(c_tma, c_reg)
    assert ogemm.rel_frobenius(c_tma.cpu(), ogemm.gemm(a.cpu(), b.cpu())) <= 1e-5
    assert opart.check_counts(counts.cpu().numpy())["ok"]
    expect = (opart.gemm_owner_map(m, n, 64, 64) if kind == tp.MAP_IDENTITY
              else opart.gemm_owner_map(m, n, 64, 64, P, "strided", group_m))
    assert np.array_equal(owner.cpu().numpy(), expect)
