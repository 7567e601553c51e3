"""Input recipes for the dust equilibrium-temperature workloads.

Everything here is input synthesis, in FP64 with numpy, seeded with PCG64:

* wavelength grid: ``K`` log-spaced wavelengths and the quadrature weights
  ``w_k = lambda_k * Delta * (1/2 at both ends)``, ``Delta = ln(lmax/lmin)/(K-1)``:
  the trapezoid rule in ln(lambda) applied to ``f(lambda) * lambda``, so that
  ``sum_k w_k f(lambda_k)`` approximates ``int f dlambda``.  This is the
  paper's "finite-difference" Delta-lambda_l of Eqs. 6-8 (Section 4), which it
  leaves unspecified.
* toy grain model: ``C_abs = pi a^2 Q`` with
  ``Q = min(1, 2 pi a / lambda) (lambda / 1um)^-beta (1 + sum_b A_b exp(-(lambda-lambda_b)^2 / (2 (rho_b lambda_b)^2)))``.
  The paper used Laor & Draine graphite cross sections (Section 5), which are
  not available; these stand in with the same shapes (sizes x wavelengths).
* heating field: a dilute two-temperature stellar blackbody mix
  ``J = U J_ISRF [0.7 B(5000 K)/int B + 0.3 B(20000 K)/int B]`` with
  ``log10 U`` uniform, optionally attenuated by ``exp(-tau_V (lambda/0.55um)^-1.3)``.
  The paper used the intensities of a simulated Sbc galaxy (Section 5); these
  stand in for them.  The blackbody here is the *input spectrum shape*; the
  method's own Planck arithmetic lives in the oracle and in the kernels.
* grain numbers: ``n[c,g] = rho_c n0_g`` with an MRN-like ``dn/dln a ~ a^-2.5``
  normalised to unit grain volume per species, and ``rho_c ~ LogNormal(0, 1)``.
  This is the paper's ``n_s m_d;c`` of Eqs. 9-10 (Section 4), generalised to
  any ``n[c,g]``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

# SI 2019 exact defining constants, used only to shape the synthetic heating field.
_H = 6.62607015e-34
_C = 299792458.0
_KB = 1.380649e-23
_SIGMA_SB = 2.0 * math.pi ** 5 * _KB ** 4 / (15.0 * _H ** 3 * _C ** 2)

UM = 1.0e-6
NM = 1.0e-9

#: Bolometric mean intensity of the local interstellar radiation field that
#: ``U = 1`` stands for [W m^-2 sr^-1] (c u / 4 pi with u ~ 8.4e-14 J m^-3).
J_ISRF = 2.0e-6

#: Toy grain species: power-law slope beta and Gaussian features
#: (centre [m], amplitude, relative width).
SPECIES = {
    "silicate": {"beta": 1.6, "bumps": [(9.7 * UM, 1.0, 0.10)]},
    "graphite": {"beta": 2.0, "bumps": [(0.2175 * UM, 1.0, 0.05)]},
    "pah": {
        "beta": 2.0,
        "bumps": [(lc * UM, 2.0, 0.02) for lc in (3.3, 6.2, 7.7, 8.6, 11.3)],
    },
}

#: The workload configurations: a tiny case, the 2^18-cell FP32 path, the same
#: shapes for the mixed-precision form, and the 2^20-cell large solve.
CONFIGS = {
    0: dict(name="tiny", n_cells=1024, K=64, lam_um=(0.09, 1000.0),
            species=("silicate", "graphite"), n_sizes=8, a_um=(0.003, 1.0),
            log10U=(-3.0, 4.0), opaque_frac=0.0, tau_V=(5.0, 50.0), seed=1000),
    1: dict(name="fp32-2^18", n_cells=1 << 18, K=200, lam_um=(0.09, 1000.0),
            species=("silicate", "graphite", "pah"), n_sizes=32, a_um=(0.00035, 1.0),
            log10U=(-3.0, 5.0), opaque_frac=0.0, tau_V=(5.0, 50.0), seed=1001),
    2: dict(name="mixed-2^18", n_cells=1 << 18, K=200, lam_um=(0.09, 1000.0),
            species=("silicate", "graphite", "pah"), n_sizes=32, a_um=(0.00035, 1.0),
            log10U=(-3.0, 5.0), opaque_frac=0.0, tau_V=(5.0, 50.0), seed=1002),
    3: dict(name="large-2^20", n_cells=1 << 20, K=500, lam_um=(0.05, 2000.0),
            species=("silicate", "graphite", "pah"), n_sizes=80, a_um=(0.00035, 1.0),
            log10U=(-4.0, 6.0), opaque_frac=0.10, tau_V=(5.0, 50.0), seed=1003),
}

T_MIN = 2.0
T_MAX = 3000.0
N_TABLE = 4096


def wavelength_grid(K: int, lam_min: float, lam_max: float):
    """Log-spaced wavelengths [m] and trapezoid-in-ln(lambda) weights [m]."""
    if K < 2:
        raise ValueError("need at least two wavelengths")
    k = np.arange(K, dtype=np.float64)
    lam = lam_min * (lam_max / lam_min) ** (k / (K - 1))
    delta = math.log(lam_max / lam_min) / (K - 1)
    w = lam * delta
    w[0] *= 0.5
    w[-1] *= 0.5
    return lam, w


def grain_table(species: Sequence[str], n_sizes: int, a_min: float, a_max: float):
    """Species index and radius [m] of every grain g (species-major order)."""
    if n_sizes == 1:
        a = np.array([a_min])
    else:
        a = a_min * (a_max / a_min) ** (np.arange(n_sizes) / (n_sizes - 1))
    sp = np.repeat(np.arange(len(species)), n_sizes)
    return sp, np.tile(a, len(species))


def cross_sections(lam: np.ndarray, species: Sequence[str], sp_of_g: np.ndarray,
                   a_of_g: np.ndarray) -> np.ndarray:
    """Absorption cross sections C_abs[g, k] [m^2] of the toy grain model."""
    G, K = len(a_of_g), len(lam)
    out = np.empty((G, K), dtype=np.float64)
    for g in range(G):
        prm = SPECIES[species[sp_of_g[g]]]
        a = a_of_g[g]
        q = np.minimum(1.0, 2.0 * math.pi * a / lam) * (lam / UM) ** (-prm["beta"])
        bump = np.ones_like(lam)
        for lc, amp, rel in prm["bumps"]:
            bump += amp * np.exp(-((lam - lc) ** 2) / (2.0 * (rel * lc) ** 2))
        out[g] = math.pi * a * a * q * bump
    return out


def blackbody_shape(lam: np.ndarray, T: float) -> np.ndarray:
    """Blackbody spectrum of temperature T normalised to unit integral over
    wavelength [m^-1]; the spectral shape of a synthetic heating field."""
    x = _H * _C / (lam * _KB * T)
    em1 = -np.expm1(-x)
    with np.errstate(over="ignore", under="ignore", divide="ignore", invalid="ignore"):
        b = 2.0 * _H * _C * _C / lam ** 5 * np.where(x < 745.0, np.exp(-x) / em1, 0.0)
    return b / (_SIGMA_SB * T ** 4 / math.pi)


def stellar_shape(lam: np.ndarray) -> np.ndarray:
    """0.7 (5000 K) + 0.3 (20000 K) energy-weighted mix, unit integral [m^-1]."""
    return 0.7 * blackbody_shape(lam, 5000.0) + 0.3 * blackbody_shape(lam, 20000.0)


def size_weights(sp_of_g: np.ndarray, a_of_g: np.ndarray) -> np.ndarray:
    """MRN-like grain numbers per unit grain volume of each species."""
    n0 = np.empty(len(a_of_g))
    for s in np.unique(sp_of_g):
        idx = np.nonzero(sp_of_g == s)[0]
        a = a_of_g[idx]
        dlna = math.log(a[-1] / a[0]) / (len(a) - 1) if len(a) > 1 else 1.0
        raw = a ** -3.5 * a * dlna
        vol = np.sum(raw * (4.0 / 3.0) * math.pi * a ** 3)
        n0[idx] = raw / vol
    return n0


@dataclasses.dataclass
class Workload:
    name: str
    lam: np.ndarray          # [K]    m
    w: np.ndarray            # [K]    m
    C_abs: np.ndarray        # [G,K]  m^2
    J: np.ndarray            # [n,K]  float32, W m^-2 m^-1 sr^-1
    n: np.ndarray            # [n,G]  float32
    T_min: float
    T_max: float
    n_table: int
    cells: np.ndarray        # global indices of the generated cells
    n_cells_total: int
    sp_of_g: np.ndarray
    a_of_g: np.ndarray
    seed: int

    @property
    def K(self) -> int:
        return len(self.lam)

    @property
    def G(self) -> int:
        return self.C_abs.shape[0]


def _cell_draws(cfg: dict, n_cells: int, seed: int):
    rng = np.random.default_rng(seed)
    log10U = rng.uniform(cfg["log10U"][0], cfg["log10U"][1], n_cells)
    rho = np.exp(rng.standard_normal(n_cells))
    opaque = rng.random(n_cells) < cfg["opaque_frac"]
    tau_V = rng.uniform(cfg["tau_V"][0], cfg["tau_V"][1], n_cells)
    return 10.0 ** log10U, rho, opaque, tau_V


def make_workload(config, cells: Optional[np.ndarray] = None, seed: Optional[int] = None,
                  chunk: int = 1 << 16) -> Workload:
    """Build workload ``config`` (an index into CONFIGS or a dict of the same keys).

    ``cells`` selects which of the config's cells to materialise (default: all);
    per-cell draws are taken from the full seeded stream, so cell ``i`` has the
    same inputs whichever subset it is generated in.
    """
    cfg = dict(CONFIGS[config]) if isinstance(config, int) else dict(config)
    seed = cfg["seed"] if seed is None else seed
    C_total = cfg["n_cells"]
    lam, w = wavelength_grid(cfg["K"], cfg["lam_um"][0] * UM, cfg["lam_um"][1] * UM)
    sp, a = grain_table(cfg["species"], cfg["n_sizes"], cfg["a_um"][0] * UM, cfg["a_um"][1] * UM)
    C_abs = cross_sections(lam, cfg["species"], sp, a)
    U, rho, opaque, tau_V = _cell_draws(cfg, C_total, seed)
    cells = np.arange(C_total) if cells is None else np.asarray(cells, dtype=np.int64)
    shape = J_ISRF * stellar_shape(lam)
    ext = (lam / (0.55 * UM)) ** -1.3
    K, G = len(lam), len(a)
    J = np.empty((len(cells), K), dtype=np.float32)
    for s in range(0, len(cells), chunk):
        idx = cells[s:s + chunk]
        blk = U[idx, None] * shape[None, :]
        op = opaque[idx]
        if op.any():
            blk[op] *= np.exp(-tau_V[idx][op, None] * ext[None, :])
        J[s:s + len(idx)] = blk
    n0 = size_weights(sp, a)
    n = (rho[cells, None] * n0[None, :]).astype(np.float32)
    return Workload(name=cfg["name"], lam=lam, w=w, C_abs=C_abs, J=J, n=n,
                    T_min=cfg.get("T_min", T_MIN), T_max=cfg.get("T_max", T_MAX),
                    n_table=cfg.get("n_table", N_TABLE), cells=cells, n_cells_total=C_total,
                    sp_of_g=sp, a_of_g=a, seed=seed)


# ---------------------------------------------------------------- serving stream
SERVE_K = (100, 200, 350, 500)
SERVE_G = {48: 16, 96: 32, 240: 80}   # grains -> sizes per species (3 species)


def serve_snapshot_config(snapshot: int, K: int, G: int, n_cells: int) -> dict:
    """Config dict of one request drawn from snapshot ``snapshot``.

    K = 500 requests use the large wavelength range and the opaque-cell mix of
    the large solve; the others the 0.09-1000 um grid of the mid-size configs.
    """
    if K not in SERVE_K or G not in SERVE_G:
        raise ValueError("unsupported request shape")
    big = K == 500
    return dict(name=f"snap{snapshot}-K{K}-G{G}", n_cells=n_cells, K=K,
                lam_um=(0.05, 2000.0) if big else (0.09, 1000.0),
                species=("silicate", "graphite", "pah"), n_sizes=SERVE_G[G],
                a_um=(0.00035, 1.0), log10U=(-4.0, 6.0) if big else (-3.0, 5.0),
                opaque_frac=0.10 if big else 0.0, tau_V=(5.0, 50.0), seed=5000 + snapshot)


def serve_requests(n_requests: int = 2000, n_snapshots: int = 64, rate_hz: float = 100.0,
                   cells_range=(1e3, 1e6), seed: int = 4242):
    """Poisson arrival stream of solve requests.

    Returns a list of dicts with arrival time [s], snapshot, K, G, n_cells.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    snaps = rng.integers(0, n_snapshots, n_requests)
    ks = rng.choice(np.array(SERVE_K), n_requests)
    gs = rng.choice(np.array(sorted(SERVE_G)), n_requests)
    lo, hi = math.log(cells_range[0]), math.log(cells_range[1])
    cells = np.exp(rng.uniform(lo, hi, n_requests)).astype(np.int64)
    return [dict(t=float(t[i]), snapshot=int(snaps[i]), K=int(ks[i]), G=int(gs[i]),
                 n_cells=int(cells[i])) for i in range(n_requests)]


# ------------------------------------------------------- fluctuating grains
#: Toy heat-capacity model of each species: an Einstein solid of N atoms with
#: one characteristic temperature theta, E(T) = 3 N k_B theta / (exp(theta/T) - 1)
#: (zero-point energy removed).  Bulk density [kg m^-3], mean mass per atom
#: [kg] and theta [K].  The paper names no heat capacity; these give the
#: enthalpy a small grain needs to be heated by one photon.
_AMU = 1.66053906660e-27
HEAT_CAPACITY = {
    "silicate": {"rho": 3500.0, "m_atom": 24.0 * _AMU, "theta": 500.0},
    "graphite": {"rho": 2240.0, "m_atom": 12.0 * _AMU, "theta": 900.0},
    "pah": {"rho": 2240.0, "m_atom": 12.0 * _AMU, "theta": 900.0},
}


def heat_capacity_params(species: Sequence[str], sp_of_g: np.ndarray, a_of_g: np.ndarray):
    """Atoms per grain and Einstein temperature of every grain g: the two
    numbers of its enthalpy E(T) = 3 N k_B theta / (exp(theta / T) - 1)."""
    N = np.empty(len(a_of_g))
    theta = np.empty(len(a_of_g))
    for g, (s, a) in enumerate(zip(sp_of_g, a_of_g)):
        prm = HEAT_CAPACITY[species[s]]
        N[g] = (4.0 / 3.0) * math.pi * a ** 3 * prm["rho"] / prm["m_atom"]
        theta[g] = prm["theta"]
    return N, theta


def fluctuating_selection(a_of_g: np.ndarray, a_min: float = 0.5 * NM, a_max: float = 10.0 * NM):
    """Indices of the grains treated as thermally fluctuating: radii in
    [a_min, a_max] (grains much smaller hold too little energy for one UV
    photon on any useful level grid, larger ones are near equilibrium)."""
    return np.nonzero((a_of_g >= a_min) & (a_of_g <= a_max))[0]
