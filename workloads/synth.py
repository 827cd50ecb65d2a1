"""Seeded synthetic workloads shaped like the five SALT photometry configurations.

This module only draws inputs: model grids, bandpass curves, ragged observation
tables and parameter samples. It holds none of the photometry arithmetic
(no interpolation, colour law, band integral or zero point). Where a workload
needs observed fluxes at the true parameters, the caller passes the model
fluxes in (``add_noise``); the bench, which may not evaluate the model on the
host, uses ``template_flux``, a model-free light-curve shape whose values do
not change the amount of work.

Every array that the GPU path reads in single precision is rounded to float32
here, so the FP64 oracle and the GPU see bit-identical inputs.

Recipes (all numpy PCG64, seed 1000 + config index unless a seed is given):
  grids   phase -20..50 step 1 d (71 nodes); wavelength 2000..9200 step 10 A
          (721 nodes), or 2000..11000 (901) for the large batch.
          M0 = 0.1 E (1 + 0.3 sum_m a_m sin(2 pi f_m u + b_m) sin(2 pi g_m v + c_m)),
          M1 = 0.01 E (zero-mean sinusoid sum); E = raised-cosine edge taper over
          3 nodes on every edge times exp(-p^2 / (2 * 15^2)).
  bands   Gaussian, peak 1, truncated at +-3 sigma, 5 A samples on multiples of 5.
  obs     mjd ~ U[t0 - 15, t0 + 45], t0 ~ U(55000, 56000); bands round-robin over
          the bands whose rest-frame span lies inside the grid at the true z.
  params  z ~ U(0.01, zmax), x1 ~ N(0, 1), c ~ N(0, 0.1),
          x0 = 1e-5 (d_L(0.1) / d_L(z))^2 in flat LCDM (Om = 0.3, H0 = 70).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

F32 = np.float32

# Colour-law coefficient draw: a_m ~ U(-0.5, 0.5) (four coefficients).
CL_RANGE = (2800.0, 7000.0)


@dataclass
class Model:
    phase0: float
    dphase: float
    n_phase: int
    wave0: float
    dwave: float
    n_wave: int
    m0: np.ndarray  # float32 [n_phase, n_wave]
    m1: np.ndarray  # float32 [n_phase, n_wave]
    cl: np.ndarray  # float64 [4]
    cl_lo: float = CL_RANGE[0]
    cl_hi: float = CL_RANGE[1]
    # non-uniform axes: ascending node positions (None = uniform axis)
    phase_nodes: np.ndarray | None = None
    wave_nodes: np.ndarray | None = None

    @property
    def phase_max(self) -> float:
        if self.phase_nodes is not None:
            return float(self.phase_nodes[-1])
        return self.phase0 + (self.n_phase - 1) * self.dphase

    @property
    def wave_max(self) -> float:
        if self.wave_nodes is not None:
            return float(self.wave_nodes[-1])
        return self.wave0 + (self.n_wave - 1) * self.dwave


@dataclass
class Band:
    wave: np.ndarray   # float64 [K], ascending
    trans: np.ndarray  # float64 [K]


@dataclass
class Batch:
    """Ragged CSR batch: supernova s owns obs[obs_off[s]:obs_off[s+1]] and
    parameter samples par[par_off[s]:par_off[s+1]]."""
    obs_off: np.ndarray  # int64 [n_sn + 1]
    mjd: np.ndarray      # float64 [n_obs]
    band: np.ndarray     # int32 [n_obs]
    flux: np.ndarray     # float32 [n_obs]
    fluxerr: np.ndarray  # float32 [n_obs]
    zp: np.ndarray       # float32 [n_obs]
    par_off: np.ndarray  # int64 [n_sn + 1]
    t0: np.ndarray       # float64 [n_par]
    z: np.ndarray        # float32 [n_par]
    x0: np.ndarray       # float32 [n_par]
    x1: np.ndarray       # float32 [n_par]
    c: np.ndarray        # float32 [n_par]
    truth: dict = field(default_factory=dict)  # per-SN true parameters

    @property
    def n_sn(self) -> int:
        return len(self.obs_off) - 1

    @property
    def n_obs(self) -> int:
        return int(self.obs_off[-1])

    @property
    def n_par(self) -> int:
        return int(self.par_off[-1])

    def n_bandflux(self) -> int:
        n = np.diff(self.obs_off)
        s = np.diff(self.par_off)
        return int(np.sum(n * s))


# ----------------------------------------------------------------------------
# grids


def _taper(n: int) -> np.ndarray:
    """Raised-cosine taper over the 3 nodes next to each end of an axis."""
    d = np.minimum(np.arange(n), np.arange(n)[::-1]).astype(np.float64)
    return 0.5 * (1.0 - np.cos(np.pi * np.minimum(d, 3.0) / 3.0))


def make_model(rng: np.random.Generator, wave_max: float = 9200.0,
               phase=(-20.0, 50.0, 1.0), wave0: float = 2000.0,
               dwave: float = 10.0) -> Model:
    p0, p1, dp = phase
    n_phase = int(round((p1 - p0) / dp)) + 1
    n_wave = int(round((wave_max - wave0) / dwave)) + 1
    p = p0 + dp * np.arange(n_phase)
    u = (np.arange(n_phase) / (n_phase - 1))[:, None]
    v = (np.arange(n_wave) / (n_wave - 1))[None, :]
    env = (_taper(n_phase) * np.exp(-p * p / (2 * 15.0 ** 2)))[:, None] * _taper(n_wave)[None, :]

    def sines(amp_bound):
        s = np.zeros((n_phase, n_wave))
        for _ in range(3):
            a = rng.uniform(-amp_bound, amp_bound)
            f, g = rng.integers(1, 4, size=2)
            b, c = rng.uniform(0, 2 * np.pi, size=2)
            s += a * np.sin(2 * np.pi * f * u + b) * np.sin(2 * np.pi * g * v + c)
        return s

    m0 = 0.1 * env * (1.0 + 0.3 * sines(1.0))
    m1 = 0.01 * env * sines(1.0)
    cl = rng.uniform(-0.5, 0.5, size=4)
    return Model(phase0=p0, dphase=dp, n_phase=n_phase, wave0=wave0, dwave=dwave,
                 n_wave=n_wave, m0=m0.astype(F32), m1=m1.astype(F32), cl=cl)


def make_model_nodes(rng: np.random.Generator, phase_nodes, wave_nodes, cl_amp: float = 0.5) -> Model:
    """Synthetic surfaces on non-uniform axes (same recipe as make_model, the
    smooth factors taken at the node positions, the edge taper over 3 nodes).
    Colour-law coefficients ~ U(-cl_amp, cl_amp): grids reaching the NIR need
    small ones, since the law continues linearly with its slope at cl_hi."""
    p = np.asarray(phase_nodes, dtype=np.float64)
    w = np.asarray(wave_nodes, dtype=np.float64)
    n_phase, n_wave = len(p), len(w)
    u = ((p - p[0]) / (p[-1] - p[0]))[:, None]
    v = ((w - w[0]) / (w[-1] - w[0]))[None, :]
    env = (_taper(n_phase) * np.exp(-p * p / (2 * 15.0 ** 2)))[:, None] * _taper(n_wave)[None, :]

    def sines(amp_bound):
        s = np.zeros((n_phase, n_wave))
        for _ in range(3):
            a = rng.uniform(-amp_bound, amp_bound)
            f, g = rng.integers(1, 4, size=2)
            b, c = rng.uniform(0, 2 * np.pi, size=2)
            s += a * np.sin(2 * np.pi * f * u + b) * np.sin(2 * np.pi * g * v + c)
        return s

    m0 = 0.1 * env * (1.0 + 0.3 * sines(1.0))
    m1 = 0.01 * env * sines(1.0)
    cl = rng.uniform(-cl_amp, cl_amp, size=4)
    return Model(phase0=float(p[0]), dphase=float(p[1] - p[0]), n_phase=n_phase, wave0=float(w[0]),
                 dwave=float(w[1] - w[0]), n_wave=n_wave, m0=m0.astype(F32), m1=m1.astype(F32), cl=cl,
                 phase_nodes=p, wave_nodes=w)


# SALT3-NIR-shaped axes: phase denser around peak; wavelength 10 A to 9200 A,
# then 40 A steps out to 20000 A.
NIR_PHASE_NODES = np.concatenate([np.arange(-20.0, -5.0, 1.0), np.arange(-5.0, 5.0, 0.5),
                                  np.arange(5.0, 50.01, 1.5)])
NIR_WAVE_NODES = np.concatenate([np.arange(2000.0, 9200.0, 10.0), np.arange(9200.0, 20000.01, 40.0)])


# ----------------------------------------------------------------------------
# bands


def gaussian_band(center: float, n_samples: int, step: float = 5.0) -> Band:
    """Gaussian transmission, peak 1, sampled every `step` A on multiples of
    `step`, spanning +-3 sigma (sigma = step (K - 1) / 6)."""
    sigma = step * (n_samples - 1) / 6.0
    start = step * round((center - 3 * sigma) / step)
    wave = start + step * np.arange(n_samples, dtype=np.float64)
    mid = start + 0.5 * step * (n_samples - 1)
    trans = np.exp(-0.5 * ((wave - mid) / sigma) ** 2)
    return Band(wave=wave, trans=trans)


def tophat_band(lo: float, hi: float, step: float = 5.0) -> Band:
    n = int(round((hi - lo) / step)) + 1
    wave = lo + step * np.arange(n, dtype=np.float64)
    return Band(wave=wave, trans=np.ones(n))


# ----------------------------------------------------------------------------
# cosmology for x0(z)


def lum_dist(z: np.ndarray, om: float = 0.3, h0: float = 70.0, steps: int = 2000) -> np.ndarray:
    """Flat LCDM luminosity distance in Mpc, Simpson's rule on `steps` intervals."""
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    out = np.empty_like(z)
    c_kms = 299792.458
    for i, zi in enumerate(z):
        x = np.linspace(0.0, zi, steps + 1)
        f = 1.0 / np.sqrt(om * (1 + x) ** 3 + 1 - om)
        w = np.ones(steps + 1)
        w[1:-1:2] = 4
        w[2:-1:2] = 2
        integral = (zi / steps) / 3.0 * np.sum(w * f)
        out[i] = (1 + zi) * c_kms / h0 * integral
    return out


def x0_of_z(z: np.ndarray) -> np.ndarray:
    zz = np.asarray(z, dtype=np.float64)
    uniq, inv = np.unique(np.round(zz, 4), return_inverse=True)
    dl = lum_dist(uniq)[inv]
    return 1e-5 * (lum_dist(np.array([0.1]))[0] / dl) ** 2


# ----------------------------------------------------------------------------
# observation tables


def valid_bands(bands, z: float, model: Model):
    out = []
    for b, band in enumerate(bands):
        lo = band.wave[0] / (1 + z)
        hi = band.wave[-1] / (1 + z)
        if lo >= model.wave0 and hi <= model.wave_max:
            out.append(b)
    return out


def make_batch(rng, model, bands, n_obs_per_sn, z_true, n_samples_per_sn,
               perturb=None, zp=27.5, fixed_bands_round_robin=True) -> Batch:
    """Draw the ragged observation table and the parameter samples.

    Observed fluxes are left at zero; fill them with ``add_noise`` (model fluxes
    at the truth) or ``template_flux``."""
    n_sn = len(n_obs_per_sn)
    z_true = np.asarray(z_true, dtype=F32).astype(np.float64)
    t0_true = rng.uniform(55000.0, 56000.0, size=n_sn)
    x1_true = rng.normal(0.0, 1.0, size=n_sn).astype(F32)
    c_true = rng.normal(0.0, 0.1, size=n_sn).astype(F32)
    x0_true = x0_of_z(z_true).astype(F32)
    obs_off = np.zeros(n_sn + 1, dtype=np.int64)
    obs_off[1:] = np.cumsum(n_obs_per_sn)
    n_obs = int(obs_off[-1])
    mjd = np.empty(n_obs)
    band = np.empty(n_obs, dtype=np.int32)
    for s in range(n_sn):
        n = int(n_obs_per_sn[s])
        vb = valid_bands(bands, z_true[s], model)
        if not vb:
            raise ValueError(f"no band inside the grid at z={z_true[s]}")
        start = rng.integers(0, len(vb))
        t = np.sort(rng.uniform(t0_true[s] - 15.0, t0_true[s] + 45.0, size=n))
        lo, hi = obs_off[s], obs_off[s + 1]
        mjd[lo:hi] = t
        band[lo:hi] = np.asarray(vb, dtype=np.int32)[(start + np.arange(n)) % len(vb)]
    par_off = np.zeros(n_sn + 1, dtype=np.int64)
    par_off[1:] = np.cumsum(n_samples_per_sn)
    sn_of_par = np.repeat(np.arange(n_sn), n_samples_per_sn)
    t0 = t0_true[sn_of_par].copy()
    z = z_true[sn_of_par].copy()
    x0 = x0_true[sn_of_par].astype(np.float64)
    x1 = x1_true[sn_of_par].astype(np.float64)
    c = c_true[sn_of_par].astype(np.float64)
    if perturb is not None:
        n_par = len(t0)
        z = np.clip(z + rng.normal(0, perturb["z"], n_par), 0.001, None)
        t0 = t0 + rng.normal(0, perturb["t0"], n_par)
        x0 = x0 * np.exp(rng.normal(0, perturb["logx0"], n_par))
        x1 = x1 + rng.normal(0, perturb["x1"], n_par)
        c = c + rng.normal(0, perturb["c"], n_par)
    truth = dict(z=z_true.astype(F32), t0=t0_true, x0=x0_true, x1=x1_true, c=c_true)
    return Batch(obs_off=obs_off, mjd=mjd, band=band,
                 flux=np.zeros(n_obs, dtype=F32), fluxerr=np.ones(n_obs, dtype=F32),
                 zp=np.full(n_obs, zp, dtype=F32), par_off=par_off, t0=t0,
                 z=z.astype(F32), x0=x0.astype(F32), x1=x1.astype(F32), c=c.astype(F32),
                 truth=truth)


def truth_batch(batch: Batch) -> Batch:
    """The same observation table with exactly one sample per SN: the truth."""
    n_sn = batch.n_sn
    return Batch(obs_off=batch.obs_off, mjd=batch.mjd, band=batch.band, flux=batch.flux,
                 fluxerr=batch.fluxerr, zp=batch.zp,
                 par_off=np.arange(n_sn + 1, dtype=np.int64),
                 t0=np.asarray(batch.truth["t0"], dtype=np.float64),
                 z=np.asarray(batch.truth["z"], dtype=F32),
                 x0=np.asarray(batch.truth["x0"], dtype=F32),
                 x1=np.asarray(batch.truth["x1"], dtype=F32),
                 c=np.asarray(batch.truth["c"], dtype=F32), truth=batch.truth)


FIT_PERTURB = dict(t0=2.0, logx0=0.1, x1=0.5, c=0.05)


def fit_start(batch: Batch, rng: np.random.Generator, perturb=None) -> Batch:
    """Starting points for fitting: the same observation table with one sample
    per SN at the truth, t0, x0, x1 and c perturbed (Gaussian; log-normal for
    x0) and z kept at the truth (a known redshift). FP32 parameters are
    rounded to FP32 here, so every consumer reads the same values."""
    p = FIT_PERTURB if perturb is None else perturb
    tb = truth_batch(batch)
    n = tb.n_sn
    t0 = tb.t0 + rng.normal(0.0, p["t0"], n)
    x0 = (tb.x0.astype(np.float64) * np.exp(rng.normal(0.0, p["logx0"], n))).astype(F32)
    x1 = (tb.x1.astype(np.float64) + rng.normal(0.0, p["x1"], n)).astype(F32)
    c = (tb.c.astype(np.float64) + rng.normal(0.0, p["c"], n)).astype(F32)
    return Batch(obs_off=tb.obs_off, mjd=tb.mjd, band=tb.band, flux=tb.flux, fluxerr=tb.fluxerr,
                 zp=tb.zp, par_off=tb.par_off, t0=t0, z=tb.z, x0=x0, x1=x1, c=c, truth=tb.truth)


def add_noise(batch: Batch, m_true: np.ndarray, rng: np.random.Generator,
              frac: float = 0.05, noiseless: bool = False) -> None:
    """Observed flux = model flux at the truth + frac-Gaussian noise.

    sigma_i = frac * max(|m_i|, 0.01 * max_SN |m|); `m_true` is supplied by the
    caller (one value per observation)."""
    m = np.asarray(m_true, dtype=np.float64)
    sig = np.empty_like(m)
    for s in range(batch.n_sn):
        lo, hi = batch.obs_off[s], batch.obs_off[s + 1]
        if hi == lo:
            continue
        mm = np.abs(m[lo:hi])
        sig[lo:hi] = frac * np.maximum(mm, 0.01 * mm.max() + 1e-300)
    f = m if noiseless else m + sig * rng.normal(0.0, 1.0, size=m.shape)
    batch.flux = f.astype(F32)
    batch.fluxerr = sig.astype(F32)


def template_flux(batch: Batch, rng: np.random.Generator, frac: float = 0.05) -> None:
    """Model-free observed fluxes: a skewed Gaussian-in-time light curve around
    the true t0 with an amplitude that scales like x0, plus frac noise. Used
    where the model may not be evaluated on the host; the values change no
    amount of work."""
    n_sn = batch.n_sn
    n = np.diff(batch.obs_off)
    sn = np.repeat(np.arange(n_sn), n)
    dt = batch.mjd - batch.truth["t0"][sn]
    width = np.where(dt < 0, 8.0, 20.0)
    amp = 2.0e13 * (batch.truth["x0"][sn].astype(np.float64) / 1e-5)
    m = amp * np.exp(-0.5 * (dt / width) ** 2) * (1.0 + 0.2 * np.cos(batch.band + 0.3))
    sig = frac * np.maximum(np.abs(m), 0.01 * amp)
    batch.flux = (m + sig * rng.normal(0.0, 1.0, size=m.shape)).astype(F32)
    batch.fluxerr = sig.astype(F32)


def subset(batch: Batch, sns) -> Batch:
    """The batch restricted to the given supernova indices (kept in order)."""
    sns = np.asarray(sns, dtype=np.int64)
    n = np.diff(batch.obs_off)[sns]
    s_cnt = np.diff(batch.par_off)[sns]
    oi = np.concatenate([np.arange(batch.obs_off[s], batch.obs_off[s + 1]) for s in sns]) \
        if len(sns) else np.zeros(0, dtype=np.int64)
    pi = np.concatenate([np.arange(batch.par_off[s], batch.par_off[s + 1]) for s in sns]) \
        if len(sns) else np.zeros(0, dtype=np.int64)
    oo = np.zeros(len(sns) + 1, dtype=np.int64)
    oo[1:] = np.cumsum(n)
    po = np.zeros(len(sns) + 1, dtype=np.int64)
    po[1:] = np.cumsum(s_cnt)
    truth = {k: np.asarray(v)[sns] for k, v in batch.truth.items()}
    return Batch(obs_off=oo, mjd=batch.mjd[oi], band=batch.band[oi], flux=batch.flux[oi],
                 fluxerr=batch.fluxerr[oi], zp=batch.zp[oi], par_off=po,
                 t0=batch.t0[pi], z=batch.z[pi], x0=batch.x0[pi], x1=batch.x1[pi],
                 c=batch.c[pi], truth=truth)


# ----------------------------------------------------------------------------
# the five workloads

PERTURB = dict(z=0.01, t0=2.0, logx0=0.05, x1=0.3, c=0.03)

CONFIG_NAMES = {
    1: "plain_1sn_40obs",
    2: "batched_chi2_1000sn",
    3: "diff_256sn_x1024",
    4: "serving_20000req",
    5: "large_ragged_100000sn_x64",
}


@dataclass
class Workload:
    name: str
    model: Model
    bands: list
    batch: Batch | None
    requests: list | None = None


def config1(seed: int = 1001) -> Workload:
    """1 SN, 40 observations over 4 bands (10 each); z=0.1, x0=1e-5, x1=0.5, c=0.05."""
    rng = np.random.default_rng(seed)
    model = make_model(rng)
    bands = [gaussian_band(c, 481) for c in (4500.0, 5500.0, 6500.0, 8000.0)]
    b = make_batch(rng, model, bands, [40], [0.1], [1])
    b.truth.update(x0=np.array([1e-5], F32), x1=np.array([0.5], F32), c=np.array([0.05], F32))
    b.x0[:] = F32(1e-5)
    b.x1[:] = F32(0.5)
    b.c[:] = F32(0.05)
    b.band[:] = np.repeat(np.arange(4, dtype=np.int32), 10)
    return Workload(CONFIG_NAMES[1], model, bands, b)


def _six_bands(rng, centres):
    ks = rng.integers(150, 301, size=len(centres))
    return [gaussian_band(c, int(k)) for c, k in zip(centres, ks)]


def config2(seed: int = 1002, n_sn: int = 1000) -> Workload:
    """n_sn SNe, obs ~ U{20..200} over 6 Gaussian bands (centres 3700-9000 A),
    z ~ U(0.01, 1.0), one parameter vector (the truth) per SN."""
    rng = np.random.default_rng(seed)
    model = make_model(rng)
    bands = _six_bands(rng, np.linspace(3700.0, 9000.0, 6))
    n_obs = rng.integers(20, 201, size=n_sn)
    z = rng.uniform(0.01, 1.0, size=n_sn)
    b = make_batch(rng, model, bands, n_obs, z, np.ones(n_sn, dtype=np.int64))
    return Workload(CONFIG_NAMES[2], model, bands, b)


def config3(seed: int = 1003, n_sn: int = 256, n_samples: int = 1024) -> Workload:
    """n_sn SNe x n_samples prior draws around the truth, obs ~ U{50..150}."""
    rng = np.random.default_rng(seed)
    model = make_model(rng)
    bands = _six_bands(rng, np.linspace(3700.0, 9000.0, 6))
    n_obs = rng.integers(50, 151, size=n_sn)
    z = rng.uniform(0.01, 1.0, size=n_sn)
    b = make_batch(rng, model, bands, n_obs, z, np.full(n_sn, n_samples, dtype=np.int64),
                   perturb=PERTURB)
    return Workload(CONFIG_NAMES[3], model, bands, b)


def config5(seed: int = 1005, n_sn: int = 100000, n_samples: int = 64) -> Workload:
    """Large ragged batch: SALT3-shaped 71x901 grid, 8 bands, obs log-U[8, 400],
    z ~ U(0.01, 2.0), n_samples draws around the truth per SN."""
    rng = np.random.default_rng(seed)
    model = make_model(rng, wave_max=11000.0)
    ks = rng.integers(150, 301, size=8)
    bands = [gaussian_band(c, int(k)) for c, k in zip(3700.0 + 900.0 * np.arange(8), ks)]
    n_obs = np.round(np.exp(rng.uniform(np.log(8), np.log(400), size=n_sn))).astype(np.int64)
    z = rng.uniform(0.01, 2.0, size=n_sn)
    b = make_batch(rng, model, bands, n_obs, z, np.full(n_sn, n_samples, dtype=np.int64),
                   perturb=PERTURB)
    return Workload(CONFIG_NAMES[5], model, bands, b)


@dataclass
class Request:
    arrival_s: float
    want_grad: bool
    batch: Batch  # one SN


def config4(seed: int = 1004, n_req: int = 20000, rate_per_s: float = 1000.0) -> Workload:
    """Serving stream: Poisson arrivals, one SN per request, obs ~ U{10..300},
    samples round(exp(U(0, ln 4096))), half chi2-only and half chi2+grad."""
    rng = np.random.default_rng(seed)
    model = make_model(rng)
    bands = _six_bands(rng, np.linspace(3700.0, 9000.0, 6))
    n_obs = rng.integers(10, 301, size=n_req)
    n_s = np.round(np.exp(rng.uniform(0.0, np.log(4096.0), size=n_req))).astype(np.int64)
    n_s = np.clip(n_s, 1, 4096)
    z = rng.uniform(0.01, 1.0, size=n_req)
    big = make_batch(rng, model, bands, n_obs, z, n_s, perturb=PERTURB)
    template_flux(big, rng)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_req)
    t = np.cumsum(gaps)
    grad = rng.random(n_req) < 0.5
    reqs = [Request(arrival_s=float(t[i]), want_grad=bool(grad[i]), batch=subset(big, [i]))
            for i in range(n_req)]
    return Workload(CONFIG_NAMES[4], model, bands, big, requests=reqs)


def config_nir(seed: int = 1006, n_sn: int = 200, n_samples: int = 4) -> Workload:
    """Non-uniform SALT3-NIR-shaped grid (66 x 991 nodes), 3 optical + 3 NIR
    Gaussian bands (centres 4500-16500 A, 5 A sampling), obs ~ U{20..120},
    z ~ U(0.01, 0.2), n_samples draws around the truth per SN; colour-law
    coefficients ~ U(-0.02, 0.02)."""
    rng = np.random.default_rng(seed)
    model = make_model_nodes(rng, NIR_PHASE_NODES, NIR_WAVE_NODES, cl_amp=0.02)
    bands = _six_bands(rng, np.array([4500.0, 6000.0, 7500.0, 10200.0, 12500.0, 16500.0]))
    n_obs = rng.integers(20, 121, size=n_sn)
    z = rng.uniform(0.01, 0.2, size=n_sn)
    b = make_batch(rng, model, bands, n_obs, z, np.full(n_sn, n_samples, dtype=np.int64),
                   perturb=PERTURB)
    return Workload("nir_nonuniform_200sn", model, bands, b)


def make(config: int, **kw) -> Workload:
    return {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}[config](**kw)
