"""Seeded synthetic workloads shaped like the paper's datasets (Table 1, Sec. 3).

The paper evaluates on gist/deep/open-images (in-distribution queries) and
t2i/laion/wit/rqa (out-of-distribution queries); none of those files exist here,
so every input is drawn from a seeded Gaussian mixture with the same n, D,
similarity (inner product on unit-norm vectors) and the ID/OOD query structure.

This module only draws random numbers and unit-normalises them (or, for the
Euclidean workloads, leaves the mixture draws raw). It holds none
of the method's arithmetic (no projection, quantisation, search or fitting) and
is the one module that both the CUDA path's tests/bench and the CPU oracle
consume.

Recipes (all draws: numpy PCG64, float64 unless stated, cast to float32 after
normalisation):

* ``isotropic``: component means ~ N(0, I_D); x = mean_c + sigma * z,
  z ~ N(0, I_D); c uniform over the components.
* ``anisotropic``: one Haar-random basis U and a spectrum s_i proportional to
  i^-1 (normalised so sum(s) = D). Means are U diag(sqrt(s)) g with g ~ N(0, I);
  the within-component noise is sigma * U diag(sqrt(s)) z. Both signal and
  noise live in the same decaying spectrum, which is what makes a d << D
  linear projection meaningful (as for deep-learning embeddings).
* ``ood queries``: query component c reuses the database mean of c and adds a
  global modality gap g ~ N(0, gap^2 I) plus a per-component offset
  xi_c ~ N(0, offs^2 I); its noise has the same spectrum but in the rotated
  basis U O (O Haar-random), so the query second moment differs from the
  database one in both mean and covariance.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Seed offsets per stream (added to the configuration number).
SEED_DATABASE = 1000
SEED_TEST_QUERIES = 2000
SEED_LEARN_QUERIES = 3000
SEED_SAMPLING = 4000
SEED_GRAPH = 5000


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def haar_orthogonal(D: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix (QR of a Gaussian with sign fix)."""
    g = rng.standard_normal((D, D))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def decaying_spectrum(D: int, power: float = 1.0) -> np.ndarray:
    s = np.arange(1, D + 1, dtype=np.float64) ** (-power)
    return s * (D / s.sum())


def unit_rows(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    nrm = np.linalg.norm(x, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return (x / nrm).astype(np.float32)


@dataclasses.dataclass
class Mixture:
    means: np.ndarray          # C x D float64
    basis: np.ndarray | None   # D x D (None => isotropic noise)
    sqrt_spec: np.ndarray | None
    sigma: float

    def sample(self, n: int, rng: np.random.Generator, chunk: int = 65536) -> np.ndarray:
        C, D = self.means.shape
        out = np.empty((n, D), dtype=np.float32)
        comp = rng.integers(0, C, size=n)
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            z = rng.standard_normal((e - s, D), dtype=np.float32)
            if self.basis is not None:
                z = (z * self.sqrt_spec.astype(np.float32)[None, :]) @ self.basis.T.astype(np.float32)
            x = self.means[comp[s:e]] + self.sigma * z.astype(np.float64)
            out[s:e] = unit_rows(x)
        return out


    def sample_torch(self, n: int, seed: int, device, chunk: int = 131072, normalize: bool = True):
        """Same recipe drawn with torch's generator on `device` (for the million-scale
        workloads; deterministic for a given device type and torch version).  normalize=False
        keeps the raw mixture draws (the Euclidean workloads)."""
        import torch
        g = torch.Generator(device=device)
        g.manual_seed(int(seed))
        C, D = self.means.shape
        means = torch.as_tensor(self.means, dtype=torch.float32, device=device)
        basis = torch.as_tensor(self.basis.T, dtype=torch.float32, device=device) if self.basis is not None else None
        sq = torch.as_tensor(self.sqrt_spec, dtype=torch.float32, device=device) if self.sqrt_spec is not None else None
        out = torch.empty((n, D), dtype=torch.float32, device=device)
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            comp = torch.randint(0, C, (e - s,), generator=g, device=device)
            z = torch.randn((e - s, D), generator=g, device=device)
            if basis is not None:
                z = (z * sq) @ basis
            x = means[comp] + self.sigma * z
            out[s:e] = x / x.norm(dim=1, keepdim=True).clamp_min(1e-30) if normalize else x
        return out


def isotropic_mixture(D: int, components: int, sigma: float, seed: int) -> Mixture:
    rng = _rng(seed)
    return Mixture(rng.standard_normal((components, D)), None, None, sigma)


def anisotropic_mixture(D: int, components: int, sigma: float, seed: int,
                        power: float = 1.0) -> Mixture:
    rng = _rng(seed)
    U = haar_orthogonal(D, rng)
    sq = np.sqrt(decaying_spectrum(D, power))
    g = rng.standard_normal((components, D))
    means = (g * sq[None, :]) @ U.T
    return Mixture(means, U, sq, sigma)


def ood_query_mixture(db: Mixture, seed: int, gap: float = 0.5, offset: float = 0.25) -> Mixture:
    """Shifted query mixture: database means + global gap + per-component offset,
    noise spectrum rotated by a Haar-random orthogonal matrix."""
    rng = _rng(seed)
    C, D = db.means.shape
    g = gap * rng.standard_normal(D)
    xi = offset * rng.standard_normal((C, D))
    O = haar_orthogonal(D, rng)
    basis = (db.basis if db.basis is not None else np.eye(D)) @ O
    sq = db.sqrt_spec if db.sqrt_spec is not None else np.ones(D)
    return Mixture(db.means + g[None, :] + xi, basis, sq, db.sigma)


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray        # n x D database (float32, unit rows)
    Q: np.ndarray        # m x D test queries
    Q_learn: np.ndarray  # learning queries (separate draw)


def make_workload(kind: str, n: int, m: int, D: int, components: int, cfg: int,
                  sigma: float = 0.3, ood: bool = False, m_learn: int | None = None,
                  name: str = "") -> Workload:
    if kind == "isotropic":
        mix = isotropic_mixture(D, components, sigma, SEED_DATABASE + cfg)
    elif kind == "anisotropic":
        mix = anisotropic_mixture(D, components, sigma, SEED_DATABASE + cfg)
    else:
        raise ValueError(kind)
    X = mix.sample(n, _rng(SEED_DATABASE + cfg + 1))
    qmix = ood_query_mixture(mix, SEED_TEST_QUERIES + cfg + 7) if ood else mix
    Q = qmix.sample(m, _rng(SEED_TEST_QUERIES + cfg))
    ml = m if m_learn is None else m_learn
    Ql = qmix.sample(ml, _rng(SEED_LEARN_QUERIES + cfg)) if ml > 0 else np.zeros((0, D), np.float32)
    return Workload(name or kind, X, Q, Ql)


# The five workload shapes (database n x D, queries, target d) of the scope table.
def workload_id_small(n: int = 10_000, m: int = 1_000) -> Workload:
    """10k x 128 isotropic mixture (100 components, sigma 0.3), ID queries."""
    return make_workload("isotropic", n, m, 128, 100, cfg=1, sigma=0.3, m_learn=0,
                         name=f"id-{n//1000}k-128")


def workload_id_large(n: int = 1_000_000, m: int = 10_000, D: int = 768,
                      components: int = 1000) -> Workload:
    """1M x 768 anisotropic mixture (1000 components, i^-1 spectrum), ID queries."""
    return make_workload("anisotropic", n, m, D, components, cfg=2, sigma=0.3, m_learn=m,
                         name=f"id-{n//1000}k-{D}")


def workload_ood(n: int = 1_000_000, m: int = 10_000, D: int = 512, components: int = 1000,
                 cfg: int = 3) -> Workload:
    """Shifted-query mixture (database n x D, OOD test + learning queries)."""
    return make_workload("anisotropic", n, m, D, components, cfg=cfg, sigma=0.3, ood=True,
                         m_learn=m, name=f"ood-{n//1000}k-{D}")


def make_workload_torch(kind: str, n: int, m: int, D: int, components: int, cfg: int, device,
                        sigma: float = 0.3, ood: bool = False, m_learn: int | None = None, normalize: bool = True):
    """make_workload drawn on a CUDA device (float32 tensors X, Q, Q_learn); normalize=False for the
    Euclidean workloads (raw mixture draws)."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        mix = (isotropic_mixture(D, components, sigma, SEED_DATABASE + cfg) if kind == "isotropic"
               else anisotropic_mixture(D, components, sigma, SEED_DATABASE + cfg))
        X = mix.sample_torch(n, SEED_DATABASE + cfg + 1, device, normalize=normalize)
        qmix = ood_query_mixture(mix, SEED_TEST_QUERIES + cfg + 7) if ood else mix
        Q = qmix.sample_torch(m, SEED_TEST_QUERIES + cfg, device, normalize=normalize)
        ml = m if m_learn is None else m_learn
        Ql = qmix.sample_torch(ml, SEED_LEARN_QUERIES + cfg, device, normalize=normalize)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return X, Q, Ql


def subsample_rows(n: int, n_s: int, cfg: int) -> np.ndarray:
    """Uniform subsample without replacement (seeded), sorted indices."""
    rng = _rng(SEED_SAMPLING + cfg)
    if n_s >= n:
        return np.arange(n)
    return np.sort(rng.choice(n, size=n_s, replace=False))


def uneven_batch(m: int, seed: int, ks=(1, 10, 100), L_range=(20, 300)) -> np.ndarray:
    """Per-query (k, L) for an uneven batch: k uniform over classes, L uniform integer
    in L_range, with L raised to at least k. Returns m x 2 int32."""
    rng = _rng(seed)
    k = np.asarray(ks)[rng.integers(0, len(ks), size=m)]
    L = rng.integers(L_range[0], L_range[1] + 1, size=m)
    L = np.maximum(L, k)
    return np.stack([k, L], axis=1).astype(np.int32)
