"""Synthetic Gaia-like catalogues (seeded).

The paper tests its mapper on simulated Gaia stars (Sale & Magorrian 2018,
Sect. 5); that catalogue is not available, so the workloads here stand in for
it.  Each workload fixes a sky field, a star count, a distance law, the
turbulence hyperparameters of the log-density GP (variance sigma2 and outer
scale L0 of a Kolmogorov spectrum truncated at the injection scale, Sect. 1)
and the noise level of the extinction observations.

Truth: a log-density field f is drawn on a 2 pc grid by spectral synthesis
with power P(k) ~ (k^2 + k0^2)^(-11/6), k0 = 1/L0, normalised to variance
sigma2 and mean ln(rho_bar) - sigma2/2 so that E[exp f] = rho_bar; the true
extinction to a star is the line integral of exp(f) from the Sun to the star
(trilinear interpolation at 2 pc steps).  The observation is
A_obs = A_true + N(0, A_sigma^2).

Nothing here evaluates the covariance or runs inference: this module only
produces input arrays.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DEG = math.pi / 180.0


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    l_deg: tuple            # (l_min, l_max) of the field, degrees
    b_deg: tuple            # (b_min, b_max) of the field, degrees
    s_pc: tuple = (100.0, 3000.0)   # distances log-uniform in this range
    sigma2: float = 1.0     # variance of the log-density GP
    outer_scale_pc: float = 20.0
    rho_bar: float = 1e-3   # mean extinction density, mag/pc (1 mag/kpc)
    cutoff_factor: float = 3.0  # sparsity cutoff = factor * outer scale
    n_nodes: int = 32       # Gauss-Legendre nodes per sightline
    noise: tuple = (0.05, 0.05)  # A_sigma uniform in this range, mag
    seed: int = 0

    @property
    def cutoff_pc(self) -> float:
        return self.cutoff_factor * self.outer_scale_pc


# The five workloads the hot path is built and measured on.  The first is
# small enough for the dense CPU oracle; the second is the throughput case.
WORKLOADS = {
    "c1_plain_400": Workload("c1_plain_400", 400, (0.0, 1.0), (0.0, 1.0),
                             n_nodes=32),
    "c2_plain_20k": Workload("c2_plain_20k", 20000, (0.0, 5.0), (0.0, 5.0),
                             n_nodes=64),
    "c3_mixed_200k": Workload("c3_mixed_200k", 200000, (0.0, 10.0),
                              (-5.0, 5.0), outer_scale_pc=10.0, n_nodes=64,
                              noise=(0.03, 0.1)),
    "c5_surrogate_1m": Workload("c5_surrogate_1m", 1000000, (0.0, 20.0),
                                (-10.0, 10.0), s_pc=(100.0, 5000.0),
                                n_nodes=64),
}


def _field_positions(rng, n, l_deg, b_deg, s_pc):
    """Uniform on the sphere inside the field; distances log-uniform."""
    l = rng.uniform(l_deg[0] * DEG, l_deg[1] * DEG, n)
    sb = rng.uniform(math.sin(b_deg[0] * DEG), math.sin(b_deg[1] * DEG), n)
    b = np.arcsin(sb)
    s = np.exp(rng.uniform(math.log(s_pc[0]), math.log(s_pc[1]), n))
    return l, b, s


def _unit(l, b):
    cb = np.cos(b)
    return np.stack([cb * np.cos(l), cb * np.sin(l), np.sin(b)], axis=-1)


def _truth_fft(rng, l, b, s, sigma2, L0, rho_bar, h=2.0, pad_factor=3.0, order=1,
               rho_fn=None):
    """Line integrals of exp(f) for a spectrally synthesised log-density f.

    order: how f is read at the integration points, 1 = trilinear
    interpolation of the grid, 0 = the value of the nearest cell.  Trilinear
    interpolation averages cells whose correlation is well below 1 (the
    Kolmogorov correlation has a cusp at zero separation: phi(0.1) = 0.8), so
    it lowers the variance of the sampled log-density and E[exp f] with it;
    nearest-cell values keep the variance sigma2.

    rho_fn: optional mean density (mag/pc) at heliocentric positions (..., 3);
    the density is then rho_fn(x) exp(f - ln rho_bar) (so E rho = rho_fn)."""
    from scipy import fft as sfft
    from scipy.ndimage import map_coordinates

    u = _unit(l, b)
    c = u.mean(axis=0)
    c /= np.linalg.norm(c)
    # orthonormal frame with e1 along the field centre
    tmp = np.array([0.0, 0.0, 1.0]) if abs(c[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    e2 = np.cross(tmp, c)
    e2 /= np.linalg.norm(e2)
    e3 = np.cross(c, e2)
    R = np.stack([c, e2, e3])              # rows: frame axes
    ends = (u * s[:, None]) @ R.T          # star positions in the frame
    pts = np.vstack([ends, np.zeros((1, 3))])
    pad = pad_factor * L0
    lo = pts.min(axis=0) - pad
    hi = pts.max(axis=0) + pad
    dims = [sfft.next_fast_len(int(math.ceil((hi[k] - lo[k]) / h)) + 2, real=True)
            for k in range(3)]
    # white noise -> filtered field (float32 to bound memory)
    w = rng.standard_normal(dims, dtype=np.float32)
    W = sfft.rfftn(w, workers=-1)
    del w
    k0 = 1.0 / L0
    kx = 2 * np.pi * sfft.fftfreq(dims[0], d=h).astype(np.float32)
    ky = 2 * np.pi * sfft.fftfreq(dims[1], d=h).astype(np.float32)
    kz = 2 * np.pi * sfft.rfftfreq(dims[2], d=h).astype(np.float32)
    k2 = (kx[:, None, None] ** 2 + ky[None, :, None] ** 2
          + kz[None, None, :] ** 2 + np.float32(k0 * k0))
    amp = k2 ** np.float32(-11.0 / 12.0)   # sqrt of P(k) ~ (k^2+k0^2)^(-11/6)
    del k2
    # variance of the synthesised field = mean over the full k-grid of amp^2;
    # the half-spectrum counts interior planes twice
    wts = np.full(amp.shape[2], 2.0, dtype=np.float64)
    wts[0] = 1.0
    if dims[2] % 2 == 0:
        wts[-1] = 1.0
    var = float((amp.astype(np.float64) ** 2).sum(axis=(0, 1)) @ wts) / np.prod(dims)
    amp *= np.float32(math.sqrt(sigma2 / var))
    W *= amp
    del amp
    f = sfft.irfftn(W, s=dims, workers=-1)
    del W
    mu_f = math.log(rho_bar) - 0.5 * sigma2
    # line integral of exp(f) at 2 pc steps (midpoint rule), trilinear interp
    A = np.empty(len(s))
    chunk = 512
    for i0 in range(0, len(s), chunk):
        idx = np.arange(i0, min(len(s), i0 + chunk))
        nst = np.ceil(s[idx] / h).astype(np.int64)
        tot = int(nst.sum())
        star = np.repeat(np.arange(len(idx)), nst)
        k = np.arange(tot) - np.repeat(np.cumsum(nst) - nst, nst)
        t0 = k * h
        t1 = np.minimum(t0 + h, s[idx][star])
        tm = 0.5 * (t0 + t1)
        ph = u[idx][star] * tm[:, None]
        p = ph @ R.T
        g = ((p - lo) / h).T
        fv = map_coordinates(f, g, order=order, mode="nearest")
        rho = np.exp(mu_f + fv) if rho_fn is None else \
            rho_fn(ph) * np.exp(mu_f - math.log(rho_bar) + fv)
        A[idx] = np.bincount(star, weights=rho * (t1 - t0), minlength=len(idx))
    return A


def make_catalogue(wl: Workload | str, n: int | None = None, seed: int | None = None,
                   truth: str = "fft"):
    """Draw a catalogue for workload `wl` (optionally overriding n and seed).

    truth='fft'  : spectral synthesis of the log-density on a 2 pc grid,
                   read by trilinear interpolation.
    truth='fft_nearest' : the same field read at the nearest cell (keeps the
                   log-density's variance; see _truth_fft).
    truth='mean' : A_true = rho_bar * s (no turbulence; fast, for unit tests).
    Returns a dict of float64 arrays l, b (radians), s (pc), A_obs, A_sigma,
    A_true (mag) plus the workload's hyperparameters.
    """
    if isinstance(wl, str):
        wl = WORKLOADS[wl]
    n = wl.n if n is None else int(n)
    seed = wl.seed if seed is None else int(seed)
    ss = np.random.SeedSequence([seed, n, 1708_09705])
    r_pos, r_truth, r_noise = [np.random.default_rng(c) for c in ss.spawn(3)]
    l, b, s = _field_positions(r_pos, n, wl.l_deg, wl.b_deg, wl.s_pc)
    if truth in ("fft", "fft_nearest"):
        A_true = _truth_fft(r_truth, l, b, s, wl.sigma2, wl.outer_scale_pc, wl.rho_bar,
                            order=1 if truth == "fft" else 0)
    elif truth == "mean":
        A_true = wl.rho_bar * s
    else:
        raise ValueError(truth)
    sig = r_noise.uniform(wl.noise[0], wl.noise[1], n) if wl.noise[1] > wl.noise[0] \
        else np.full(n, wl.noise[0])
    A_obs = A_true + sig * r_noise.standard_normal(n)
    return dict(l=l, b=b, s=s, A_obs=A_obs, A_sigma=sig, A_true=A_true,
                sigma2=wl.sigma2, outer_scale_pc=wl.outer_scale_pc,
                rho_bar=wl.rho_bar, cutoff_pc=wl.cutoff_pc, n_nodes=wl.n_nodes,
                name=wl.name, seed=seed)


# Sect. 5 set-up: an exponential disc of dust plus a Gaussian bump (a spiral
# arm) along the line of sight.  Parameters of the truth (L, H, rho0, s_bump,
# A_bump in pc, pc, mag/pc, pc, mag); Sun at 8 kpc from the Galactic centre;
# bump width 400 pc.
DISC_TRUTH = (2500.0, 150.0, 0.9e-3, 2200.0, 0.15)
R_SUN_PC, BUMP_WIDTH_PC = 8000.0, 400.0


def disc_density(x, theta=DISC_TRUTH):
    """Mean pseudo-density of the Sect. 5 truth at heliocentric positions x
    (pc, x-axis towards the Galactic centre)."""
    L, H, rho0, sb, Ab = theta
    R = np.hypot(R_SUN_PC - x[..., 0], x[..., 1])
    d = np.linalg.norm(x, axis=-1)
    return (rho0 * np.exp(-(R - R_SUN_PC) / L - np.abs(x[..., 2]) / H)
            + Ab / (BUMP_WIDTH_PC * math.sqrt(2 * math.pi))
            * np.exp(-0.5 * ((d - sb) / BUMP_WIDTH_PC) ** 2))


def make_disc_catalogue(n=6000, seed=0, theta=DISC_TRUTH, sigma_lnA=0.05, truth="fft",
                        l_deg=(174.0, 186.0), b_deg=(-2.5 / 60, 2.5 / 60),
                        s_pc=(100.0, 5000.0), outer_scale_pc=20.0, sigma2=1.0):
    """The Sect. 5 letter-box field towards the anticentre (174 <= l < 186
    deg, |b| < 2.5 arcmin, distances to 5 kpc) with the disc-plus-bump mean
    density `theta` and a log-density GP on top; observations of the
    log-extinction with Gaussian noise sigma_lnA (the simplified case of
    Sect. 4.1).  truth='fft' synthesises the fluctuations (nearest-cell
    reading), truth='mean' uses the mean extinction only (a numerical line
    integral of the mean density, 1 pc steps)."""
    wl = Workload("sect5_disc", n, l_deg, b_deg, s_pc=s_pc, sigma2=sigma2,
                  outer_scale_pc=outer_scale_pc, n_nodes=64, seed=seed)
    ss = np.random.SeedSequence([seed, n, 5])
    r_pos, r_truth, r_noise = [np.random.default_rng(c) for c in ss.spawn(3)]
    l, b, s = _field_positions(r_pos, n, wl.l_deg, wl.b_deg, wl.s_pc)
    rho_fn = lambda x: disc_density(x, theta)
    if truth == "fft":
        A_true = _truth_fft(r_truth, l, b, s, sigma2, outer_scale_pc, wl.rho_bar, order=0,
                            rho_fn=rho_fn)
    elif truth == "mean":
        u = _unit(l, b)
        A_true = np.empty(n)
        for i in range(n):
            t = (np.arange(int(math.ceil(s[i]))) + 0.5) * (s[i] / math.ceil(s[i]))
            A_true[i] = rho_fn(u[i] * t[:, None]).sum() * (s[i] / math.ceil(s[i]))
    else:
        raise ValueError(truth)
    sig = np.full(n, float(sigma_lnA))
    a_obs = np.log(A_true) + sig * r_noise.standard_normal(n)
    return dict(l=l, b=b, s=s, A_obs=a_obs, A_sigma=sig, A_true=A_true, sigma2=sigma2,
                outer_scale_pc=outer_scale_pc, rho_bar=wl.rho_bar, cutoff_pc=wl.cutoff_pc,
                n_nodes=wl.n_nodes, name=wl.name, seed=seed, theta_true=np.array(theta),
                r_sun_pc=R_SUN_PC, bump_width_pc=BUMP_WIDTH_PC)


def catalogue_subset(cat, idx):
    """Rows `idx` of a catalogue dict (hyperparameters kept)."""
    out = dict(cat)
    for k in ("l", "b", "s", "A_obs", "A_sigma", "A_true"):
        out[k] = np.asarray(cat[k])[idx]
    return out


def make_fields(n_fields=256, n_range=(500, 8000), side_deg=(1.0, 3.0),
                L0_range=(10.0, 40.0), seed=0, truth="mean", scale=1.0):
    """Independent fields for the batched workload: star counts log-uniform in
    n_range (times `scale`), square fields with side uniform in side_deg,
    outer scales uniform in L0_range.  Fields are spread in longitude so they
    never overlap.  Returns a list of catalogue dicts."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, n_fields, 4]))
    out = []
    for f in range(n_fields):
        nf = max(1, int(round(scale * math.exp(rng.uniform(math.log(n_range[0]),
                                                            math.log(n_range[1]))))))
        side = rng.uniform(*side_deg)
        L0 = rng.uniform(*L0_range)
        l0 = (f * 5.0) % 360.0
        wl = Workload(f"field{f}", nf, (l0, l0 + side), (-side / 2, side / 2),
                      outer_scale_pc=L0, n_nodes=64, seed=seed * 100003 + f)
        out.append(make_catalogue(wl, truth=truth))
    return out
