"""Seeded synthetic workloads for the two-level LPBF heat solve.

This module only describes inputs: domain and mesh sizes, material
constants, process parameters and laser scan paths.  It holds none of the
method's arithmetic (no interpolation, no laser position along a path, no
assembly), so that both the CUDA path and the CPU oracle can take their
inputs from here without sharing any computation.

The shapes mirror the paper's 3D experiments (Section 5.2 single track,
Section 5.3 alternating multi-track scan on a bare plate): a coarse global
mesh of uniform hexahedra, a fine local patch at the top surface that follows
the laser, a time ratio m between macro and micro steps.  The paper's IN625
property curves are not available, so the material is a Ti64-like alloy with
linear c(T), k(T); powder is the top 50 um layer with 1 % of the solid
conductivity until it melts.

A workload is a plain dict whose keys are the fields of ``tl_config``
(declared in ``include/tl.h``) plus ``macro_steps`` and ``name``.
"""
from __future__ import annotations

import copy

import numpy as np

# Material and process constants shared by every workload (SI units).
MATERIAL = dict(
    rho=4430.0,          # kg/m^3
    c0=526.0, c1=0.15,   # c(T) = c0 + c1 (T - Tref)   J/(kg K)
    k0=6.7, k1=0.011,    # k(T) = k0 + k1 (T - Tref)   W/(m K)
    Tref=293.0,
    powder_depth=50e-6,  # m, top layer that starts as powder
    powder_factor=0.01,  # k_powder = powder_factor * k_solid
    T_melt=1900.0,       # K, powder consolidates above this element-mean T
    latent=0.0,          # J/kg, latent heat of fusion (0: off; Ti64 ~ 2.86e5)
    T_solidus=1878.0,    # K, phase-change sigmoid centred at (T_solidus + T_liquidus) / 2
    T_liquidus=1923.0,   # K
    pc_sharpness=0.05,   # 1/K, sigmoid sharpness S
)
PROCESS = dict(P=195.0, eta=0.4, radius=50e-6)
THERMAL = dict(T0=293.0, T_bottom=293.0)
# top-surface losses (Section 3.1): off in every workload unless overridden
SURFACE = dict(h_conv=0.0, emissivity=0.0, T_amb=293.0)
SOLVER = dict(precision=0, tol=1e-12, tol_inner=1e-5, max_iter=2000, inner_tiles=0,
              coupling_sweeps=1, coupling_tol=1e-10, precond=0, coarse_source=0, bc_weight_literal=0, energy=1,
              picard_iters=1)


def raster_tracks(x_start, x_end, y_center, n_tracks, hatch, speed):
    """Alternating raster along x, tracks centred on ``y_center``.

    Track j runs from ``x_start`` to ``x_end`` when j is even and back when j
    is odd, at y = y_center + (j - (n_tracks - 1) / 2) * hatch.  Zero turn
    time between tracks.
    """
    tracks = []
    for j in range(n_tracks):
        y = y_center + (j - (n_tracks - 1) / 2.0) * hatch
        if j % 2 == 0:
            tracks.append((x_start, y, x_end, y, speed))
        else:
            tracks.append((x_end, y, x_start, y, speed))
    return tracks


def _base(**kw):
    cfg = {}
    cfg.update(MATERIAL)
    cfg.update(PROCESS)
    cfg.update(THERMAL)
    cfg.update(SURFACE)
    cfg.update(SOLVER)
    cfg.update(kw)
    return cfg


def single_track_tiny():
    """2 x 1 x 0.5 mm plate, 16x8x4 coarse hexes (125 um), 4x4x2 coarse patch
    refined 4x (16x16x8 fine), m = 4, 50 macro steps of 50 us, one track
    along x at y = 0.5 mm at 0.8 m/s."""
    return _base(
        name="single_track_tiny",
        Lx=2e-3, Ly=1e-3, Lz=0.5e-3, NXc=16, NYc=8, NZc=4,
        pNXc=4, pNYc=4, pNZc=2, r=4, m=4, dt_coarse=50e-6,
        tracks=[(0.0, 0.5e-3, 2e-3, 0.5e-3, 0.8)],
        macro_steps=50,
    )


def multitrack_10mm():
    """10 x 5 x 2 mm plate, 80x40x16 coarse hexes, 8x8x4 coarse patch refined
    8x (64x64x32 fine = 131072 elements, 65x65x33 nodes), m = 8, 2000 macro
    steps of 50 us; 10 alternating tracks of 8 mm, hatch 100 um, 0.8 m/s."""
    return _base(
        name="multitrack_10mm",
        Lx=10e-3, Ly=5e-3, Lz=2e-3, NXc=80, NYc=40, NZc=16,
        pNXc=8, pNYc=8, pNZc=4, r=8, m=8, dt_coarse=50e-6,
        tracks=raster_tracks(1e-3, 9e-3, 2.5e-3, 10, 100e-6, 0.8),
        macro_steps=2000,
    )


def multitrack_20mm():
    """20 x 10 x 4 mm plate, 160x80x32 coarse hexes, 16x16x8 coarse patch
    refined 8x (128x128x64 fine = 1048576 elements), m = 8, 50 us macro
    steps; 10 alternating tracks of 18 mm, hatch 100 um.  Timed for 200
    macro steps (the full scan is 4500)."""
    return _base(
        name="multitrack_20mm",
        Lx=20e-3, Ly=10e-3, Lz=4e-3, NXc=160, NYc=80, NZc=32,
        pNXc=16, pNYc=16, pNZc=8, r=8, m=8, dt_coarse=50e-6,
        tracks=raster_tracks(1e-3, 19e-3, 5e-3, 10, 100e-6, 0.8),
        macro_steps=200, precision=1, tol=1e-10,
    )


def probe_256():
    """Roofline probe: a 256 x 256 x 128-element fine patch (8.5M nodes, a
    working set above the 129 MB L2): 32 x 32 x 16 coarse elements refined 8x
    on a 5 x 5 x 2.5 mm plate of 40 x 40 x 20 coarse hexes, m = 8, one 3 mm
    track."""
    return _base(
        name="probe_256",
        Lx=5e-3, Ly=5e-3, Lz=2.5e-3, NXc=40, NYc=40, NZc=20,
        pNXc=32, pNYc=32, pNZc=16, r=8, m=8, dt_coarse=50e-6,
        tracks=[(1e-3, 2.5e-3, 4e-3, 2.5e-3, 0.8)],
        macro_steps=4, precision=1, tol=1e-10,
    )


def batch_jobs(n_jobs=64, seed=20211025):
    """Independent jobs of uneven size: domain length 2-8 mm (width L/2,
    depth L/4), P 100-300 W, speed 0.4-1.5 m/s, 1-6 tracks, refinement 4 or
    8 (m = r), fine patch extents drawn in [32, 96]^2 x [32, 48] elements and
    clamped to the domain.  Uniform draws from numpy default_rng(seed)."""
    rng = np.random.default_rng(seed)
    hc = 125e-6
    jobs = []
    for j in range(n_jobs):
        L = rng.uniform(2e-3, 8e-3)
        NXc = max(4, int(round(L / hc)))
        NYc = max(2, int(round(L / 2 / hc)))
        NZc = max(2, int(round(L / 4 / hc)))
        r = int(rng.choice([4, 8]))
        fx = int(rng.integers(32, 97))
        fy = int(rng.integers(32, 97))
        fz = int(rng.integers(32, 49))
        pNXc = min(NXc, max(1, fx // r))
        pNYc = min(NYc, max(1, fy // r))
        pNZc = min(NZc - 1, max(1, fz // r))
        P = rng.uniform(100.0, 300.0)
        v = rng.uniform(0.4, 1.5)
        nt = int(rng.integers(1, 7))
        Lx, Ly, Lz = NXc * hc, NYc * hc, NZc * hc
        tracks = raster_tracks(0.25 * Lx, 0.75 * Lx, 0.5 * Ly, nt, 100e-6, v)
        scan_time = nt * 0.5 * Lx / v
        dt = 50e-6
        cfg = _base(
            name=f"batch_job_{j}",
            Lx=Lx, Ly=Ly, Lz=Lz, NXc=NXc, NYc=NYc, NZc=NZc,
            pNXc=pNXc, pNYc=pNYc, pNZc=pNZc, r=r, m=r, dt_coarse=dt,
            tracks=tracks, macro_steps=int(np.ceil(scan_time / dt)),
            precision=1, tol=1e-10,
        )
        cfg["P"] = P
        jobs.append(cfg)
    return jobs


def serving_arrivals(rate=20.0, duration=60.0, seed=20211026, large_frac=0.1):
    """Poisson arrival times and job shapes for a request stream: each job is
    drawn like ``batch_jobs`` and, with probability ``large_frac``, replaced
    by the 20 mm multi-track shape truncated to its 200 timed macro steps."""
    rng = np.random.default_rng(seed)
    t = 0.0
    arrivals = []
    pool = batch_jobs(256, seed=seed + 1)
    big = multitrack_20mm()
    i = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        if rng.uniform() < large_frac:
            job = copy.deepcopy(big)
            job["name"] = f"serve_large_{i}"
        else:
            job = copy.deepcopy(pool[i % len(pool)])
            job["name"] = f"serve_job_{i}"
        arrivals.append((t, job))
        i += 1
    return arrivals


WORKLOADS = {
    "single_track_tiny": single_track_tiny,
    "multitrack_10mm": multitrack_10mm,
    "multitrack_20mm": multitrack_20mm,
    "probe_256": probe_256,
}


def workload(name, **overrides):
    """A fresh copy of a named workload with fields overridden."""
    cfg = WORKLOADS[name]()
    cfg.update(overrides)
    return cfg


def fine_nodes(cfg):
    """Node count of the fine patch."""
    r = cfg["r"]
    return ((cfg["pNXc"] * r + 1) * (cfg["pNYc"] * r + 1) * (cfg["pNZc"] * r + 1))
