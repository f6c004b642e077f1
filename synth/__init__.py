"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA-side tests/bench.

This module holds no arithmetic of the method under test (no beta-divergence, no powers,
no contractions of the updates).  Ground-truth low-rank tensors are built with
``numpy.einsum`` as plain data synthesis.  Every array that leaves this module is rounded
to float32 (and returned as float64 holding float32 values), so the FP64 oracle and the
FP32 device path see bit-identical inputs.

Workloads (all seeded with numpy's PCG64):
  * cp_dense(dims, R, ...)      -- dense CP data; "uniform_poisson" (factors U(0.1,1),
                                   model rescaled to mean 10, then Poisson) or
                                   "gamma_noise" (factors Gamma(2,1), times i.i.d.
                                   Gamma(10, 0.1) multiplicative noise).
  * tucker_dense(dims, J, ...)  -- dense Tucker data; Gamma(2,1) core and factors,
                                   rescaled to mean 10, then Poisson.
  * coo_counts(dims, nnz, ...)  -- sparse count tensor: first mode with a 7-periodic
                                   profile, second with a 24-periodic profile, last two
                                   Zipf(1.1) over seeded rank permutations, values
                                   1 + Geometric(0.3) (failures before the first success);
                                   unique coordinates, returned in random order.
  * init_factors(dims, R)       -- U(0.1, 1) initial factors (and core).
  * serving_jobs(n_jobs, ...)   -- the mixed-job request stream.
"""
import numpy as np


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _cp_model(factors):
    letters = "abcdefgh"
    spec = ",".join(f"{letters[n]}r" for n in range(len(factors))) + "->" + letters[: len(factors)]
    return np.einsum(spec, *factors, optimize=True)


def _tucker_model(core, factors):
    letters = "abcdefgh"
    upper = "ABCDEFGH"
    N = len(factors)
    spec = upper[:N] + "," + ",".join(f"{letters[n]}{upper[n]}" for n in range(N)) + "->" + letters[:N]
    return np.einsum(spec, core, *factors, optimize=True)


def init_factors(dims, R, seed=1, low=0.1, high=1.0):
    g = rng(seed)
    return [_f32(g.uniform(low, high, size=(d, R))) for d in dims]


def init_tucker(dims, J, seed=1, low=0.1, high=1.0):
    g = rng(seed)
    core = _f32(g.uniform(low, high, size=tuple(J)))
    factors = [_f32(g.uniform(low, high, size=(d, j))) for d, j in zip(dims, J)]
    return core, factors


def cp_dense(dims, R, seed=0, kind="uniform_poisson", mean_scale=10.0):
    """Dense nonnegative CP data.  Returns (X, true_factors), X float32-valued."""
    g = rng(seed)
    if kind == "uniform_poisson":
        A = [g.uniform(0.1, 1.0, size=(d, R)) for d in dims]
        M = _cp_model(A)
        M *= mean_scale / M.mean()
        X = g.poisson(M).astype(np.float64)
    elif kind == "gamma_noise":
        A = [g.gamma(2.0, 1.0, size=(d, R)) for d in dims]
        M = _cp_model(A)
        X = M * g.gamma(10.0, 0.1, size=M.shape)
    elif kind == "exact":
        A = [g.uniform(0.1, 1.0, size=(d, R)) for d in dims]
        X = _cp_model(A)
    else:
        raise ValueError(kind)
    return _f32(X), [_f32(a) for a in A]


def tucker_dense(dims, J, seed=0, mean_scale=10.0, kind="poisson"):
    """Dense nonnegative Tucker data.  Returns (X, true_core, true_factors)."""
    g = rng(seed)
    core = g.gamma(2.0, 1.0, size=tuple(J))
    A = [g.gamma(2.0, 1.0, size=(d, j)) for d, j in zip(dims, J)]
    M = _tucker_model(core, A)
    if kind == "poisson":
        M *= mean_scale / M.mean()
        X = g.poisson(M).astype(np.float64)
    elif kind == "exact":
        X = M
    else:
        raise ValueError(kind)
    return _f32(X), _f32(core), [_f32(a) for a in A]


def coo_counts(dims=(183, 24, 1140, 1717), nnz=3_300_000, seed=0, zipf_s=1.1):
    """Sparse 4-way count tensor with periodic / Zipf coordinate marginals.

    Returns (idx: list of N int32 arrays, vals: float64 array of float32 values)."""
    g = rng(seed)
    N = len(dims)
    assert N >= 2
    probs = []
    periods = [7.0, 24.0]
    for n, d in enumerate(dims):
        if n < 2:
            phase = g.uniform(0, 2 * np.pi)
            t = np.arange(d)
            w = 1.0 + 0.5 * np.sin(2 * np.pi * t / periods[n] + phase)
        else:
            ranks = g.permutation(d) + 1.0
            w = ranks ** (-zipf_s)
        probs.append(w / w.sum())
    keys = np.empty(0, dtype=np.int64)
    strides = np.cumprod([1] + list(dims[::-1]))[::-1][1:]  # row-major strides
    total = int(np.prod(dims))
    assert nnz <= total
    got = np.empty(0, dtype=np.int64)
    while got.size < nnz:
        need = int((nnz - got.size) * 1.3) + 1024
        cols = [g.choice(d, size=need, p=p).astype(np.int64) for d, p in zip(dims, probs)]
        k = np.zeros(need, dtype=np.int64)
        for n in range(N):
            k += cols[n] * strides[n]
        keys = np.concatenate([got, k])
        _, first = np.unique(keys, return_index=True)
        got = keys[np.sort(first)]
    got = got[:nnz]
    got = got[g.permutation(nnz)]
    idx = []
    rem = got.copy()
    for n in range(N):
        idx.append((rem // strides[n]).astype(np.int32))
        rem = rem % strides[n]
    failures = g.geometric(0.3, size=nnz).astype(np.float64) - 1.0  # numpy counts trials
    vals = 1.0 + failures
    return idx, _f32(vals)


def coo_from_dense(X):
    nz = np.nonzero(X)
    return [a.astype(np.int32) for a in nz], X[nz].astype(np.float64)


def serving_jobs(n_jobs, seed=0, dim_lo=16, dim_hi=256, rank_lo=4, rank_hi=32,
                 betas=(0.5, 1.0, 1.5), rate=None):
    """Mixed request stream: per job model (CP or Tucker), dims log-uniform in
    [dim_lo, dim_hi], rank / core dims uniform in [rank_lo, rank_hi], beta from `betas`,
    Poisson arrival times at `rate` jobs/s (None: all at t=0), and a data seed."""
    g = rng(seed)
    jobs = []
    t = 0.0
    for q in range(n_jobs):
        model = "cp" if g.uniform() < 0.5 else "tucker"
        dims = tuple(int(round(np.exp(g.uniform(np.log(dim_lo), np.log(dim_hi))))) for _ in range(3))
        if model == "cp":
            rank = int(g.integers(rank_lo, rank_hi + 1))
            J = None
        else:
            J = tuple(int(g.integers(rank_lo, rank_hi + 1)) for _ in range(3))
            J = tuple(min(j, d) for j, d in zip(J, dims))
            rank = None
        beta = float(betas[int(g.integers(0, len(betas)))])
        if rate:
            t += g.exponential(1.0 / rate)
        jobs.append(dict(id=q, model=model, dims=dims, rank=rank, core=J, beta=beta, arrival=t,
                         seed=int(g.integers(0, 2**31 - 1))))
    return jobs


def job_data(job):
    """Data and init for one serving job: Poisson-noised low-rank model at mean 10."""
    if job["model"] == "cp":
        X, _ = cp_dense(job["dims"], job["rank"], seed=job["seed"], kind="uniform_poisson")
        A0 = init_factors(job["dims"], job["rank"], seed=job["seed"] + 1)
        return X, None, A0
    X, _, _ = tucker_dense(job["dims"], job["core"], seed=job["seed"])
    G0, A0 = init_tucker(job["dims"], job["core"], seed=job["seed"] + 1)
    return X, G0, A0


def job_data_torch(job, device="cuda"):
    """Same recipe as job_data, drawn on the device with a seeded torch generator (used to
    feed the serving benchmark without host-side generation of large jobs)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(job["seed"]))
    dims = job["dims"]
    if job["model"] == "cp":
        R = job["rank"]
        A = [torch.rand((d, R), generator=g, device=device) * 0.9 + 0.1 for d in dims]
        M = torch.einsum("ir,jr,kr->ijk", *A)
        M *= 10.0 / M.mean()
        X = torch.poisson(M, generator=g).float()
        A0 = [torch.rand((d, R), generator=g, device=device) * 0.9 + 0.1 for d in dims]
        return X.contiguous(), None, [a.contiguous() for a in A0]
    J = job["core"]
    core = torch.distributions.Gamma(torch.full(tuple(J), 2.0, device=device), 1.0).sample()
    A = [torch.rand((d, j), generator=g, device=device) * 2.0 for d, j in zip(dims, J)]
    M = torch.einsum("abc,ia,jb,kc->ijk", core, *A)
    M *= 10.0 / M.mean()
    X = torch.poisson(M, generator=g).float()
    G0 = torch.rand(tuple(J), generator=g, device=device) * 0.9 + 0.1
    A0 = [torch.rand((d, j), generator=g, device=device) * 0.9 + 0.1 for d, j in zip(dims, J)]
    return X.contiguous(), G0.contiguous(), [a.contiguous() for a in A0]
