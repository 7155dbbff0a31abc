"""Seeded synthetic sparse tensors for sparse FastTucker SGD.

This module only makes inputs: COO index arrays, values, initial factor and
core matrices and sample permutations.  Both the CUDA path and the FP64 oracle
consume what it returns; it holds no step of the SGD method itself.  The one
piece of model arithmetic here is the evaluation of a *planted* model (to make
values that have a known low-rank structure), written with plain torch ops and
used for nothing else.

Randomness comes from one counter-based generator, SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): draw i of
stream k under seed S is mix64(key(S, k) + (i + 1) * 0x9E3779B97F4A7C15).  It is
written with wrapping int64 torch ops, so a tensor drawn on the CPU and one
drawn on a GPU are bit-identical, and a large workload can be made directly in
device memory.

Workload shapes follow the paper's experiments (Section "Experimental
Settings"): a Netflix-shaped ratings tensor (480000 x 17800 x 2200, skewed user
and item modes, integer ratings 1-5), Synthetic(Order)-style uniform tensors of
order 3-10 with equal mode lengths, and Synthetic(Sparsity)-style order-3
tensors.  The public datasets themselves are not used; only their shapes and
value ranges are.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
import torch

_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _s64(c: int) -> int:
    """Unsigned 64-bit constant -> the int64 with the same bits."""
    c &= _MASK64
    return c - (1 << 64) if c >= (1 << 63) else c


def _srl(x: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bits."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def mix64(x: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output function on int64 tensors (wrapping arithmetic)."""
    x = (x ^ _srl(x, 30)) * _s64(_M1)
    x = (x ^ _srl(x, 27)) * _s64(_M2)
    return x ^ _srl(x, 31)


def mix64_int(x: int) -> int:
    """The same function on Python ints (used to derive stream keys)."""
    x &= _MASK64
    x = ((x ^ (x >> 30)) * _M1) & _MASK64
    x = ((x ^ (x >> 27)) * _M2) & _MASK64
    return x ^ (x >> 31)


def stream_key(seed: int, *path: int) -> int:
    """Key of a named sub-stream: folds (seed, path...) through mix64."""
    k = mix64_int(seed * _GOLDEN + 0x632BE59BD9B4E019)
    for p in path:
        k = mix64_int(k ^ mix64_int((p + 1) * _GOLDEN))
    return k


def bits(key: int, n: int, offset: int = 0, device="cpu") -> torch.Tensor:
    """n raw 64-bit draws (as int64) of the stream with the given key."""
    i = torch.arange(offset + 1, offset + n + 1, dtype=torch.int64, device=device)
    return mix64(i * _s64(_GOLDEN) + _s64(key))


def uniform(key: int, n: int, offset: int = 0, device="cpu") -> torch.Tensor:
    """Float64 uniforms in [0, 1) from the top 53 bits of each draw."""
    return _srl(bits(key, n, offset, device), 11).to(torch.float64) * (2.0 ** -53)


def normal(key: int, n: int, offset: int = 0, device="cpu") -> torch.Tensor:
    """Float64 standard normals by the Box-Muller transform of two streams."""
    u1 = uniform(key ^ 0x1, n, offset, device)
    u2 = uniform(key ^ 0x2, n, offset, device)
    return torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * math.pi * u2)


def permutation(key: int, n: int, device="cpu") -> torch.Tensor:
    """Seeded permutation of range(n) (argsort of draws), int64."""
    return torch.argsort(bits(key, n, 0, device), stable=True)


def zipf_ranks(key: int, n: int, support: int, s: float, offset: int = 0, device="cpu"):
    """n draws of a Zipf(s) rank in [0, support) by inverse CDF."""
    w = np.arange(1, support + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cdf_t = torch.from_numpy(cdf).to(device)
    u = uniform(key, n, offset, device)
    r = torch.searchsorted(cdf_t, u, right=True)
    return torch.clamp(r, max=support - 1)


@dataclasses.dataclass
class TensorSpec:
    """Shape, value law and model sizes of one synthetic workload."""
    name: str
    dims: Sequence[int]
    nnz: int
    J: Sequence[int]
    R: int
    index_law: Sequence[str]          # per mode: "uniform" or "zipf"
    zipf_s: float = 1.1
    values: str = "planted"           # "planted" (real values) or "ratings" (integers 1..5)
    planted_sigma: float = 0.3        # std of planted factor / core entries
    noise_sigma: float = 0.0
    test_fraction: float = 0.0
    init: str = "planted_law"         # "planted_law" or "uniform_mean"
    seed: int = 0

    @property
    def order(self) -> int:
        return len(self.dims)


def spec_small(seed: int = 0) -> TensorSpec:
    """Order-3 1000x800x600, 200k distinct uniform nonzeros, planted J=R=8
    model with N(0, 0.3^2) entries plus N(0, 0.01^2) noise."""
    return TensorSpec("order3-1000x800x600-200k-J8R8", (1000, 800, 600), 200_000, (8, 8, 8), 8,
                      ("uniform",) * 3, values="planted", planted_sigma=0.3, noise_sigma=0.01,
                      seed=seed)


def spec_ratings(nnz: int = 100_000_000, seed: int = 0,
                 dims=(480_000, 17_800, 2_200)) -> TensorSpec:
    """Netflix-shaped ratings tensor: user and item modes Zipf(1.1) with a
    seeded rank->id scatter, time mode uniform, integer values 1-5 from a
    standardised planted J=R=16 model, 90/10 train/test split."""
    return TensorSpec(f"ratings-{dims[0]}x{dims[1]}x{dims[2]}-{nnz}-J16R16", tuple(dims), nnz,
                      (16, 16, 16), 16, ("zipf", "zipf", "uniform"), zipf_s=1.1, values="ratings",
                      planted_sigma=0.3, noise_sigma=0.0, test_fraction=0.1, init="uniform_mean",
                      seed=seed)


def spec_order(order: int = 8, dim: int = 10_000, nnz: int = 50_000_000, J: int = 32,
               seed: int = 0) -> TensorSpec:
    """Synthetic(Order)-style uniform tensor with a planted J=R model whose
    entry std is chosen so that std(x) is about 1, plus N(0, 0.05^2) noise."""
    # std(x) = sqrt(R) * (sqrt(J) sigma^2)^N = 1  ->  sigma = (R^(-1/(2N)) / sqrt(J))^(1/2)
    sigma = math.sqrt(J ** (-0.5) * J ** (-1.0 / (2 * order)))
    return TensorSpec(f"order{order}-{dim}-{nnz}-J{J}R{J}", (dim,) * order, nnz, (J,) * order, J,
                      ("uniform",) * order, values="planted", planted_sigma=sigma,
                      noise_sigma=0.05, seed=seed)


def spec_sparsity(nnz: int, seed: int = 0, dim: int = 1000, J: int = 16) -> TensorSpec:
    """Synthetic(Sparsity)-style tensor: order 3, every mode `dim` long, `nnz`
    distinct uniform nonzeros (20M..100M at dim 1000 is 2%..10% dense), integer
    values 1-5 from a standardised planted J=R model, 90/10 split, init as the
    ratings tensor."""
    return TensorSpec(f"sparsity-{dim}^3-{nnz}-J{J}R{J}", (dim,) * 3, nnz, (J,) * 3, J,
                      ("uniform",) * 3, values="ratings", planted_sigma=0.3, noise_sigma=0.0,
                      test_fraction=0.1, init="uniform_mean", seed=seed)


def spec_batch(count: int = 64, seed: int = 0, dims=(1_000, 200_000), nnz=(10_000, 5_000_000),
               orders=(3, 6), ranks=(4, 8, 16, 32)) -> List[TensorSpec]:
    """Independent problems for the batched runner: order uniform in
    [orders[0], orders[1]], each I_n and nnz log-uniform in the given ranges
    (nnz at most a quarter of prod I_n), J_n = R drawn from `ranks`, uniform
    distinct indices, planted model with std(x) ~ 1 (entry std as
    spec_order) plus N(0, 0.01^2) noise."""
    out = []
    for i in range(count):
        u = uniform(stream_key(seed, 30, i), 12).tolist()
        N = orders[0] + min(int(u[0] * (orders[1] - orders[0] + 1)), orders[1] - orders[0])
        R = ranks[min(int(u[1] * len(ranks)), len(ranks) - 1)]
        lo, hi = math.log(dims[0]), math.log(dims[1])
        ds = tuple(int(round(math.exp(lo + (hi - lo) * u[2 + k]))) for k in range(N))
        total = 1
        for d in ds:
            total *= d
        nlo, nhi = math.log(nnz[0]), math.log(nnz[1])
        nz = int(round(math.exp(nlo + (nhi - nlo) * u[10])))
        nz = max(1, min(nz, total // 4))
        sigma = math.sqrt(R ** -0.5 * R ** (-1.0 / (2 * N)))
        out.append(TensorSpec(f"batch{i}-order{N}-R{R}-{nz}", ds, nz, (R,) * N, R,
                              ("uniform",) * N, values="planted", planted_sigma=sigma,
                              noise_sigma=0.01, seed=stream_key(seed, 31, i) & 0x7fffffff))
    return out


def _draw_indices(spec: TensorSpec, n: int, rnd: int, device) -> List[torch.Tensor]:
    out = []
    for k, (I, law) in enumerate(zip(spec.dims, spec.index_law)):
        key = stream_key(spec.seed, 1, k, rnd)
        if law == "uniform":
            u = uniform(key, n, 0, device)
            out.append(torch.clamp((u * I).to(torch.int64), max=I - 1))
        elif law == "zipf":
            r = zipf_ranks(key, n, I, spec.zipf_s, 0, device)
            scatter = permutation(stream_key(spec.seed, 2, k), I, device)
            out.append(scatter[r])
        else:
            raise ValueError(law)
    return out


def _distinct_indices(spec: TensorSpec, device) -> List[torch.Tensor]:
    """nnz distinct index tuples.  Exact linear keys when prod(I) < 2^62;
    otherwise the expected number of duplicates nnz^2 / (2 prod I) is below
    1e-9 and no dedup is done."""
    N = spec.order
    total = 1
    for I in spec.dims:
        total *= I
    if total >= (1 << 62):
        return _draw_indices(spec, spec.nnz, 0, device)
    strides = []
    acc = 1
    for I in reversed(spec.dims):
        strides.append(acc)
        acc *= I
    strides = list(reversed(strides))
    if spec.nnz > total:
        raise ValueError("more nonzeros than cells")
    keys = torch.empty(0, dtype=torch.int64, device=device)
    rnd = 0
    while keys.numel() < spec.nnz:
        need = spec.nnz - keys.numel()
        draw = need + need // 8 + 1024
        idx = _draw_indices(spec, draw, rnd, device)
        k = torch.zeros(draw, dtype=torch.int64, device=device)
        for i, st in zip(idx, strides):
            k += i * st
        keys = torch.unique(torch.cat([keys, k]))
        rnd += 1
        if rnd > 200:
            raise RuntimeError("could not draw enough distinct nonzeros")
    if keys.numel() > spec.nnz:
        pick = permutation(stream_key(spec.seed, 3), keys.numel(), device)[: spec.nnz]
        keys = keys[pick]
    # storage order: one seeded shuffle (the fixed traversal order of the tensor)
    keys = keys[permutation(stream_key(spec.seed, 4), keys.numel(), device)]
    out = []
    for st, I in zip(strides, spec.dims):
        out.append((keys // st) % I)
    return out


def planted_values(idx: Sequence[torch.Tensor], U: Sequence[torch.Tensor],
                   chunk: int = 1 << 22) -> torch.Tensor:
    """Values of a planted rank-R model at the given coordinates:
    sum_r prod_k U[k][i_k, r] (float64; U[k] = A_planted[k] @ B_planted[k])."""
    n = idx[0].numel()
    out = torch.empty(n, dtype=torch.float64, device=idx[0].device)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        prod = None
        for k in range(len(U)):
            rows = U[k][idx[k][c0:c1]]
            prod = rows if prod is None else prod * rows
        out[c0:c1] = prod.sum(dim=1)
    return out


@dataclasses.dataclass
class SparseTensor:
    """A synthetic workload: COO nonzeros (int32 SoA indices, float32 values),
    its train/test split, and the initial parameters (float32)."""
    spec: TensorSpec
    idx: List[torch.Tensor]          # train indices, int32, one per mode
    val: torch.Tensor                # train values, float32
    test_idx: List[torch.Tensor]
    test_val: torch.Tensor
    A0: List[torch.Tensor]           # initial factor matrices I_n x J_n, float32
    B0: List[torch.Tensor]           # initial core matrices J_n x R, float32

    @property
    def nnz(self) -> int:
        return int(self.val.numel())


def make_tensor(spec: TensorSpec, device="cpu") -> SparseTensor:
    """Build the workload described by ``spec`` on ``device``."""
    N, R = spec.order, spec.R
    idx64 = _distinct_indices(spec, device)
    # planted parameters
    Ap, Bp = [], []
    for k in range(N):
        Ap.append(spec.planted_sigma * normal(stream_key(spec.seed, 10, k), spec.dims[k] * spec.J[k],
                                              0, device).view(spec.dims[k], spec.J[k]))
        Bp.append(spec.planted_sigma * normal(stream_key(spec.seed, 11, k), spec.J[k] * R, 0,
                                              device).view(spec.J[k], R))
    U = [Ap[k] @ Bp[k] for k in range(N)]
    m = planted_values(idx64, U)
    del U, Ap, Bp
    if spec.values == "planted":
        x = m
        if spec.noise_sigma > 0:
            x = x + spec.noise_sigma * normal(stream_key(spec.seed, 12), m.numel(), 0, device)
    elif spec.values == "ratings":
        z = (m - m.mean()) / m.std()
        x = torch.clamp(torch.round(3.0 + z), 1.0, 5.0)
    else:
        raise ValueError(spec.values)
    val = x.to(torch.float32)
    idx = [i.to(torch.int32) for i in idx64]
    del idx64
    n_test = int(round(spec.test_fraction * spec.nnz))
    n_train = spec.nnz - n_test
    tr_idx = [i[:n_train].contiguous() for i in idx]
    te_idx = [i[n_train:].contiguous() for i in idx]
    tr_val, te_val = val[:n_train].contiguous(), val[n_train:].contiguous()
    # initial parameters (independent streams)
    A0, B0 = [], []
    if spec.init == "planted_law":
        for k in range(N):
            A0.append((spec.planted_sigma * normal(stream_key(spec.seed, 20, k),
                                                   spec.dims[k] * spec.J[k], 0, device))
                      .view(spec.dims[k], spec.J[k]).to(torch.float32))
            B0.append((spec.planted_sigma * normal(stream_key(spec.seed, 21, k), spec.J[k] * R, 0,
                                                   device)).view(spec.J[k], R).to(torch.float32))
    elif spec.init == "uniform_mean":
        # U(0, u) with E[x^] = mean(x): R * prod_k (J_k u^2 / 4) = mean  (one u for all entries)
        mean = float(tr_val.to(torch.float64).mean()) if n_train else 1.0
        logu = (math.log(mean) - math.log(R) - sum(math.log(j / 4.0) for j in spec.J)) / (2 * N)
        u = math.exp(logu)
        for k in range(N):
            A0.append((u * uniform(stream_key(spec.seed, 20, k), spec.dims[k] * spec.J[k], 0,
                                   device)).view(spec.dims[k], spec.J[k]).to(torch.float32))
            B0.append((u * uniform(stream_key(spec.seed, 21, k), spec.J[k] * R, 0, device))
                      .view(spec.J[k], R).to(torch.float32))
    else:
        raise ValueError(spec.init)
    return SparseTensor(spec, tr_idx, tr_val, te_idx, te_val, A0, B0)


def pass_permutation(seed: int, epoch: int, phase: int, mode: int, n: int, device="cpu"):
    """Sample order of one pass: a fresh seeded permutation per
    (epoch, phase, mode); phase 0 = factor module, 1 = core module.  uint32
    values are returned in an int32 tensor (n < 2^31)."""
    return permutation(stream_key(seed, 100, epoch, phase, mode), n, device).to(torch.int32)


def csf_order(idx, n: int) -> torch.Tensor:
    """Visit order of the paper's B-CSF traversal for mode n (Section "Tensor
    Storage Format"): the nonzeros sorted by i_n, then by the other modes'
    coordinates in ascending mode order (lexicographically), as a CSF tree
    rooted at mode n is walked.  Returned like pass_permutation (int32
    tensor holding the uint32 permutation, on the device of idx).  Only an
    ordering of the input: it carries none of the method's arithmetic."""
    N = len(idx)
    keys = [n] + [k for k in range(N) if k != n]
    order = torch.arange(idx[0].numel(), device=idx[0].device, dtype=torch.int64)
    # successive stable sorts from the least significant key to the most
    for k in reversed(keys):
        _, o = torch.sort(idx[k][order], stable=True)
        order = order[o]
    return order.to(torch.int32)
