"""Seeded synthetic workloads for the streaming Tucker update.

Layout contract: a slice of a d-way stream is an (n_1, ..., n_{d-1}) array stored column-major
(mode 1 fastest), the matricization convention of the paper (Sec. 2.1). NumPy arrays returned here
are Fortran-contiguous with the shape in paper order; ``to_rowmajor_view`` gives the equivalent
C-contiguous array with the shape reversed, which is what a row-major torch tensor holds.

Workloads (the paper's own datasets, the HCCI run and the sine-wave coefficients, are not
available; these seeded stand-ins follow the shapes and structure of its experiments, Sec. 5):

* ``LowRankStream`` -- exact multilinear-rank core times random orthonormal factors plus i.i.d.
  Gaussian noise (the exact-rank test workload: 3-way 24x20x16 slices, ranks (4,4,3,6), 40 steps,
  noise 1e-4, and the 64 uneven streams of the batched form).
* ``BlobField`` -- sums of anisotropic Gaussian blobs advected with constant velocities on a
  periodic grid, several variables per point, plus 1e-5 relative noise: a combustion-like field of
  the HCCI shape class (2-3 spatial modes x variables x time, Sec. 5.2) whose ranks grow, then
  plateau.
* ``SineWave`` -- the paper's sine-wave tensor (Sec. 5.1) with seeded N(0,1) coefficients, which
  the paper leaves unspecified.

Nothing in this module performs a step of the streaming Tucker method: it draws random numbers
and evaluates closed-form fields.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 230816395


def to_rowmajor_view(a: np.ndarray) -> np.ndarray:
    """Return the C-contiguous view (reversed shape) of a Fortran-contiguous array."""
    assert a.flags.f_contiguous
    return a.T


def _rng(*key: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([BASE_SEED, *[int(k) for k in key]]))


def random_orthonormal(rng: np.random.Generator, m: int, r: int) -> np.ndarray:
    """m x r matrix with orthonormal columns: Q of a Gaussian matrix, signs fixed so diag(R) > 0."""
    g = rng.standard_normal((m, r))
    q, rr = np.linalg.qr(g)
    s = np.sign(np.diag(rr))
    s[s == 0] = 1.0
    return q * s[None, :]


def _multi_ttm(core: np.ndarray, mats: list[np.ndarray]) -> np.ndarray:
    """core x_1 mats[0] x_2 mats[1] ... (synthesis of a Tucker-form test tensor)."""
    out = core
    for k, a in enumerate(mats):
        out = np.moveaxis(np.tensordot(a, out, axes=([1], [k])), 0, k)
    return out


# --------------------------------------------------------------------------------------------
# Exact low-rank stream
# --------------------------------------------------------------------------------------------

@dataclass
class LowRankStream:
    """X = G x_1 A_1 ... x_d A_d + N with G ~ N(0,1), A_k random orthonormal.

    ``spatial`` are n_1..n_{d-1}; ``ranks`` has d entries (the last is the streaming-mode rank);
    ``steps`` is the number of time steps n_d. Noise per slice is i.i.d. Gaussian scaled so that
    ||N_t|| = noise * ||Xbar_t|| (``noise_scope='slice'``), or over the whole tensor so that
    ||N|| = noise * ||Xbar|| (``noise_scope='tensor'``).
    """

    spatial: tuple
    ranks: tuple
    steps: int
    noise: float
    seed: int = 0
    noise_scope: str = "slice"
    dtype: type = np.float64
    core: np.ndarray = field(init=False, repr=False)
    factors: list = field(init=False, repr=False)

    def __post_init__(self):
        d = len(self.spatial) + 1
        assert len(self.ranks) == d
        rng = _rng(1, self.seed)
        self.core = rng.standard_normal(tuple(self.ranks))
        dims = list(self.spatial) + [self.steps]
        self.factors = [random_orthonormal(rng, dims[k], self.ranks[k]) for k in range(d)]
        self._noise_scale = None
        if self.noise_scope == "tensor":
            # ||Xbar||_F over all steps, and ||Z||_F of the drawn noise over all steps
            xb2 = 0.0
            z2 = 0.0
            for t in range(self.steps):
                xb2 += float(np.sum(self.signal(t) ** 2))
                z2 += float(np.sum(self._raw_noise(t) ** 2))
            self._noise_scale = self.noise * math.sqrt(xb2) / math.sqrt(z2) if z2 > 0 else 0.0

    @property
    def d(self) -> int:
        return len(self.spatial) + 1

    def signal(self, t: int) -> np.ndarray:
        mats = list(self.factors[:-1]) + [self.factors[-1][t : t + 1, :]]
        x = _multi_ttm(self.core, mats)
        return np.asfortranarray(x.reshape(self.spatial, order="F"))

    def _raw_noise(self, t: int) -> np.ndarray:
        n = int(np.prod(self.spatial))
        z = _rng(2, self.seed, t).standard_normal(n)
        return z.reshape(self.spatial, order="F")

    def slice(self, t: int) -> np.ndarray:
        """Slice t (0-based) as a Fortran-contiguous (n_1..n_{d-1}) array."""
        x = self.signal(t)
        if self.noise > 0:
            z = self._raw_noise(t)
            if self.noise_scope == "tensor":
                s = self._noise_scale
            else:
                zn = float(np.linalg.norm(z))
                s = self.noise * float(np.linalg.norm(x)) / zn if zn > 0 else 0.0
            x = x + s * z
        return np.asfortranarray(x.astype(self.dtype))

    def tensor(self, t0: int, t1: int) -> np.ndarray:
        """Slices t0..t1-1 stacked along the last mode (Fortran-contiguous)."""
        out = np.empty(tuple(self.spatial) + (t1 - t0,), dtype=self.dtype, order="F")
        for t in range(t0, t1):
            out[..., t - t0] = self.slice(t)
        return out


CONFIG1 = dict(spatial=(24, 20, 16), ranks=(4, 4, 3, 6), steps=40, noise=1e-4, tau=1e-3,
               n_init=10, seed=1, noise_scope="tensor")


def config1_tensor():
    """The plain-FP64 exact-rank workload: 24x20x16 slices, 40 steps, ranks (4,4,3,6)."""
    c = CONFIG1
    return LowRankStream(c["spatial"], c["ranks"], c["steps"], c["noise"], seed=c["seed"],
                         noise_scope=c["noise_scope"])


# --------------------------------------------------------------------------------------------
# Advected anisotropic Gaussian blobs
# --------------------------------------------------------------------------------------------

@dataclass
class BlobField:
    """f_v(x, t) = sum_b a_{b,v} exp(-1/2 delta^T Sigma_b^{-1} delta), delta = x - c_b - v_b t.

    x lies on a periodic [0,1)^3 grid of ``grid`` points (delta is the minimum image);
    c_b ~ U[0,1)^3, v_b ~ U[-0.5,0.5]^3 / ``vel_div`` per step, Sigma_b = R diag(s^2) R^T with
    s_i ~ U[0.02, 0.10] and R a random rotation, a_{b,v} ~ N(0,1). A slice is the
    (grid[0], grid[1], grid[2], nvar) tensor at one t, plus i.i.d. Gaussian noise scaled to
    ``noise`` * ||signal_t||.
    """

    grid: tuple = (192, 192, 96)
    nvar: int = 12
    nblobs: int = 40
    vel_div: float = 300.0
    noise: float = 1e-5
    seed: int = 2

    def __post_init__(self):
        rng = _rng(3, self.seed)
        nb = self.nblobs
        self.centres = rng.random((nb, 3))
        self.vel = (rng.random((nb, 3)) - 0.5) / self.vel_div
        self.sig = 0.02 + 0.08 * rng.random((nb, 3))
        prec = np.empty((nb, 3, 3))
        for b in range(nb):
            g = rng.standard_normal((3, 3))
            q, r = np.linalg.qr(g)
            q = q * np.sign(np.diag(r))[None, :]
            if np.linalg.det(q) < 0:
                q[:, 0] = -q[:, 0]
            prec[b] = q @ np.diag(1.0 / self.sig[b] ** 2) @ q.T
        self.prec = prec
        self.amp = rng.standard_normal((nb, self.nvar))

    @property
    def spatial(self) -> tuple:
        return tuple(self.grid) + (self.nvar,)

    @property
    def numel(self) -> int:
        return int(np.prod(self.spatial))

    def signal_torch(self, t: int, device="cpu", dtype=None):
        """Signal at step t as a row-major torch tensor of shape (nvar, n3, n2, n1)."""
        import torch

        dtype = dtype or torch.float64
        n1, n2, n3 = self.grid
        x = torch.arange(n1, device=device, dtype=dtype) / n1
        y = torch.arange(n2, device=device, dtype=dtype) / n2
        z = torch.arange(n3, device=device, dtype=dtype) / n3
        amp = torch.as_tensor(self.amp, device=device, dtype=dtype)  # (nb, nvar)
        out = torch.zeros((self.nvar, n3, n2, n1), device=device, dtype=dtype)
        for b in range(self.nblobs):
            c = self.centres[b] + self.vel[b] * t
            dx = x - float(c[0])
            dy = y - float(c[1])
            dz = z - float(c[2])
            dx = dx - torch.round(dx)
            dy = dy - torch.round(dy)
            dz = dz - torch.round(dz)
            p = self.prec[b]
            X = dx[None, None, :]
            Yy = dy[None, :, None]
            Z = dz[:, None, None]
            q = (float(p[0, 0]) * X * X + float(p[1, 1]) * Yy * Yy + float(p[2, 2]) * Z * Z
                 + 2.0 * float(p[0, 1]) * X * Yy + 2.0 * float(p[0, 2]) * X * Z
                 + 2.0 * float(p[1, 2]) * Yy * Z)
            g = torch.exp(-0.5 * q)
            # blob b's contribution to every variable, accumulated blob by blob
            out.addcmul_(amp[b].view(-1, 1, 1, 1), g.unsqueeze(0))
        return out.contiguous()

    def slice(self, t: int, dtype=np.float32) -> np.ndarray:
        """Slice t on the CPU: Fortran-contiguous (n1, n2, n3, nvar) array, noise from NumPy."""
        sig = self.signal_torch(t).numpy()  # (nvar, n3, n2, n1) row-major == column-major paper order
        z = _rng(4, self.seed, t).standard_normal(sig.shape)
        zn = float(np.linalg.norm(z))
        s = self.noise * float(np.linalg.norm(sig)) / zn if zn > 0 else 0.0
        out = (sig + s * z).astype(dtype)
        return out.T  # Fortran-contiguous, paper-order shape

    def slice_torch(self, t: int, device, dtype=None, gen_dtype=None):
        """Slice t generated with torch on ``device`` (noise from a torch generator seeded by t).

        Same recipe as :meth:`slice` (the noise values differ: torch and NumPy draw different
        streams); used where generating every slice on the host would be too slow.
        """
        import torch

        dtype = dtype or torch.float32
        gen_dtype = gen_dtype or torch.float64
        sig = self.signal_torch(t, device=device, dtype=gen_dtype)
        g = torch.Generator(device=device)
        g.manual_seed(BASE_SEED * 7 + 1000003 * self.seed + t)
        z = torch.randn(sig.shape, generator=g, device=device, dtype=gen_dtype)
        s = self.noise * torch.linalg.vector_norm(sig) / torch.linalg.vector_norm(z)
        return (sig + s * z).to(dtype).contiguous()


CONFIG2 = dict(grid=(192, 192, 96), nvar=12, nblobs=40, steps=300, tau=1e-4, n_init=10,
               noise=1e-5, seed=2)
CONFIG5 = dict(grid=(384, 384, 256), nvar=4, nblobs=80, steps=500, tau=1e-4, n_init=10,
               noise=1e-5, seed=5)


# --------------------------------------------------------------------------------------------
# Sine-wave tensor (Sec. 5.1)
# --------------------------------------------------------------------------------------------

@dataclass
class SineWave:
    """f(x) = sum_j c_j sin(pi (j . x)), |j_k| <= f_k, sampled on a uniform grid of [-1,1]^d.

    The exact mode-k rank is 2 f_k + 1 (Sec. 5.1). The stream has ``2 * steps_each`` slices on
    one time grid of [-1, 1]; the first block keeps only the terms with |j_k| <= ``freqs_a``, the
    second all terms with |j_k| <= ``freqs_b`` (same coefficients), so the ranks are freqs_a-based
    up to the middle and 2 freqs_b + 1 overall: the rank bump of Sec. 5.1. c_j ~ N(0,1) (seeded; the
    paper leaves them unspecified); noise is i.i.d. Gaussian scaled to ``noise`` * ||signal_t|| per
    slice.
    """

    n: tuple = (100, 100)
    steps_each: int = 2500
    freqs_a: tuple = (5, 5, 5)
    freqs_b: tuple = (5, 5, 7)
    noise: float = 1e-3
    seed: int = 6

    def __post_init__(self):
        rng = _rng(5, self.seed)
        self.c = rng.standard_normal(tuple(2 * f + 1 for f in self.freqs_b))

    @property
    def steps(self) -> int:
        return 2 * self.steps_each

    @property
    def spatial(self) -> tuple:
        return tuple(self.n)

    @staticmethod
    def _grid(m: int) -> np.ndarray:
        return np.linspace(-1.0, 1.0, m)

    def signal(self, t: int) -> np.ndarray:
        freqs = self.freqs_a if t < self.steps_each else self.freqs_b
        sl = tuple(slice(fb - f, fb + f + 1) for f, fb in zip(freqs, self.freqs_b))
        c = self.c[sl].astype(np.complex128)
        tt = self._grid(self.steps)[t]
        # sin(pi * sum_k j_k x_k) = Im(prod_k exp(i pi j_k x_k)): evaluate as a complex Tucker form
        mats = []
        for k, m in enumerate(self.n):
            j = np.arange(-freqs[k], freqs[k] + 1)
            mats.append(np.exp(1j * np.pi * np.outer(self._grid(m), j)))
        jt = np.arange(-freqs[-1], freqs[-1] + 1)
        mats.append(np.exp(1j * np.pi * tt * jt)[None, :])
        x = _multi_ttm(c, mats).imag
        return np.asfortranarray(x.reshape(self.spatial, order="F"))

    def slice(self, t: int, dtype=np.float64) -> np.ndarray:
        x = self.signal(t)
        if self.noise > 0:
            z = _rng(6, self.seed, t).standard_normal(x.shape)
            zn = float(np.linalg.norm(z))
            x = x + (self.noise * float(np.linalg.norm(x)) / zn) * z
        return np.asfortranarray(x.astype(dtype))


# --------------------------------------------------------------------------------------------
# 64 uneven streams (batched form)
# --------------------------------------------------------------------------------------------

def batched_streams(nstreams: int = 64, steps: int = 100, size_range=(32, 160),
                    rank_range=(4, 24), noise: float = 1e-4, seed: int = 4,
                    taus=(1e-2, 1e-3, 1e-4), dtype=np.float32):
    """Independent 3-way-spatial low-rank-plus-noise streams of uneven sizes, ranks and tolerances.

    Returns a list of (LowRankStream, tau) pairs.
    """
    rng = _rng(7, seed)
    out = []
    for i in range(nstreams):
        n = tuple(int(v) for v in rng.integers(size_range[0], size_range[1] + 1, size=3))
        r = [int(v) for v in rng.integers(rank_range[0], rank_range[1] + 1, size=4)]
        r = tuple(min(r[k], n[k]) if k < 3 else min(r[k], steps) for k in range(4))
        tau = float(taus[int(rng.integers(0, len(taus)))])
        s = LowRankStream(n, r, steps, noise, seed=1000 + i, noise_scope="slice", dtype=dtype)
        out.append((s, tau))
    return out
