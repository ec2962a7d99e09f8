"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only: sound-speed maps, source wavelets,
receiver layouts, initial pulses and relaxation-rate draws.  It contains none
of the lattice-Boltzmann arithmetic, so both the CUDA path and the FP64 oracle
can be fed from it without sharing any of the method's code.

All randomness comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 20240601


def gaussian_pulse(nx, ny, cx, cy, width, amp):
    """p0(x, y) = amp * exp(-r^2 / (2 width^2)) centred on node (cx, cy)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r2 = (x - cx) ** 2 + (y - cy) ** 2
    return (amp * np.exp(-r2 / (2.0 * width * width))).astype(np.float64)


def ricker(nt, fc, t0=0.0):
    """Source wavelet of the paper's Eq. (source)/(tau), sampled at t = t0 + n.

    S(t) = -(1 - 4 xi^2) exp(-2 xi^2),  xi = (2 pi fc / 3)(t - 3 / (2 fc)),
    with fc the central frequency in cycles per time step.
    """
    t = t0 + np.arange(nt, dtype=np.float64)
    xi = (2.0 * math.pi * fc / 3.0) * (t - 3.0 / (2.0 * fc))
    return -(1.0 - 4.0 * xi * xi) * np.exp(-2.0 * xi * xi)


def uniform_map(nx, ny, c=1.0):
    return np.full((ny, nx), c, dtype=np.float32)


def two_layer(nx, ny, c_top=1.0, c_bottom=2.0, split=None):
    """Two-layer medium, contrast c_top : c_bottom at row ``split`` (default mid-depth)."""
    split = ny // 2 if split is None else split
    c = np.full((ny, nx), c_top, dtype=np.float32)
    c[split:, :] = c_bottom
    return c


def random_medium(nx, ny, seed, c_lo=0.4, c_hi=1.0):
    """Smooth-free random heterogeneous medium (each site independent)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(c_lo, c_hi, size=(ny, nx)).astype(np.float32)


def block_model(nx, ny, bx0, by0, bw, bh, c_bg=1.0, c_block=1.0 / 3.0):
    """Homogeneous background with a rectangular slow block (grid-refinement workload)."""
    c = np.full((ny, nx), c_bg, dtype=np.float32)
    c[by0:by0 + bh, bx0:bx0 + bw] = np.float32(c_block)
    return c


def layered_fault_model(nx, ny, seed, n_layers=20, c_lo=1500.0, c_hi=5500.0, n_faults=4,
                        max_slope=0.1, dip_deg=(45.0, 85.0), throw=(20.0, 200.0)):
    """Layered model with dipping interfaces and normal faults.

    n_layers - 1 interface depths uniform in (0, ny), sorted; each interface has a
    slope uniform in [-max_slope, max_slope]; layer speeds uniform in [c_lo, c_hi];
    ``n_faults`` faults with x position uniform in (0, nx), dip angle uniform in
    ``dip_deg`` and throw uniform in ``throw`` cells (hanging wall shifted down).
    """
    rng = np.random.default_rng(seed)
    depths = np.sort(rng.uniform(0, ny, size=n_layers - 1))
    slopes = rng.uniform(-max_slope, max_slope, size=n_layers - 1)
    speeds = rng.uniform(c_lo, c_hi, size=n_layers)
    fx = rng.uniform(0, nx, size=n_faults)
    fdip = np.deg2rad(rng.uniform(dip_deg[0], dip_deg[1], size=n_faults))
    fthrow = rng.uniform(throw[0], throw[1], size=n_faults)
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    ye = np.repeat(y, nx, axis=1)
    for k in range(n_faults):
        hanging = x > fx[k] + y / np.tan(fdip[k])
        np.subtract(ye, fthrow[k], out=ye, where=hanging)
    layer = np.zeros((ny, nx), dtype=np.int16)
    for k in range(n_layers - 1):
        layer += ye > depths[k] + slopes[k] * (x - nx / 2.0)
    return speeds[layer].astype(np.float32)


def line_receivers(n, y, x_start, x_span):
    """n receivers on row y at x = x_start + floor(i * x_span / n)."""
    i = np.arange(n, dtype=np.int64)
    xs = x_start + (i * x_span) // n
    return np.stack([xs, np.full(n, y)], axis=1).astype(np.int32)


def ring_receivers(cx, cy, r, angles_deg):
    pts = [(int(round(cx + r * math.cos(math.radians(a)))),
            int(round(cy + r * math.sin(math.radians(a))))) for a in angles_deg]
    return np.asarray(pts, dtype=np.int32)


def mrt_rates(Q, seed, lo=0.5, hi=1.9):
    """Relaxation rates drawn uniformly in (lo, hi), arranged on the diagonal of S.

    D2Q5 S = diag(s_rho, s_v, s_v, s_e, s_p); D2Q9 S = diag(s_rho, s_v, s_v, s_e,
    s_p, s_eps, s_q, s_q, s_p) (the structure given with Eq. MRT-LB basic).
    """
    rng = np.random.default_rng(seed)
    if Q == 5:
        s_rho, s_v, s_e, s_p = rng.uniform(lo, hi, size=4)
        return [s_rho, s_v, s_v, s_e, s_p]
    s_rho, s_v, s_e, s_p, s_eps, s_q = rng.uniform(lo, hi, size=6)
    return [s_rho, s_v, s_v, s_e, s_p, s_eps, s_q, s_q, s_p]


# --- the five workloads -------------------------------------------------------------

# Two-layer workload: the source sits in the slow layer (c = 1, c_ref = 2, so
# eta = 0.5 and the D2Q5 lattice sound speed is 0.5/sqrt(2) = 0.35355 cells/step).
# A central wavelength of nx/30 cells therefore means fc = 0.35355 / (nx/30)
# cycles per step; for nx = 4096 that is 1/386.2.
TWO_LAYER_FC_4096 = 0.5 / math.sqrt(2.0) / (4096.0 / 30.0)


def two_layer_workload(n=4096, lattice=5, collision="bgk", seed=DEFAULT_SEED + 2, nrec=512,
                       sponge=40, sigma_max=0.1):
    """The 4096^2 two-layer workload (scaled to n^2 when n differs).

    Returns a dict of plain inputs: c_map, c_ref, source (x, y, wavelet), receivers,
    tau / s, w_ref, sponge settings and the step count of the full run.
    """
    scale = n / 4096.0
    c = two_layer(n, n, 1.0, 2.0)
    fc = TWO_LAYER_FC_4096 / scale
    nt = 5000
    src = (n // 2, n // 4, ricker(nt, fc))
    rec = line_receivers(nrec, n // 4, int(round(40 * scale)), n - 2 * int(round(40 * scale)))
    d = dict(nx=n, ny=n, c_map=c, c_ref=2.0, source=src, receivers=rec, steps=nt,
             lattice=lattice, collision=collision, tau=0.5, sponge_width=int(round(sponge * scale))
             if sponge else 0, sponge_sigma_max=sigma_max, periodic=False,
             w_ref=(0.0, 0.01, 0.24) if lattice == 9 else (4 / 9, 1 / 9, 1 / 36))
    if collision == "mrt":
        d["s"] = mrt_rates(lattice, seed)
    return d


def refined_block_workload(n=2048, nrec=256, steps=4000):
    """Grid-refinement workload: coarse n^2 grid (eta = 1 background), a slow block
    (c = c_ref / 3) of 448/2048 n coarse cells at the centre, covered by a refined
    patch of n/4 coarse cells (= n/2 fine cells) with a margin of n/64 coarse cells;
    Ricker source at (n/4, n/2); receivers on the line y = n/2 crossing the patch.
    Central wavelength 32/2048 n coarse cells in the background."""
    s = n / 2048.0
    bw = int(round(448 * s))
    b0 = (n - bw) // 2
    margin = max(1, int(round(32 * s)))
    nxp = bw + 2 * margin
    x0 = b0 - margin
    c = block_model(n, n, b0, b0, bw, bw, 1.0, 1.0 / 3.0)
    fc = (0.5 ** 0.5) / (32.0 * s)
    src = (n // 4, n // 2, ricker(steps, fc))
    lo, hi = n // 8, n - n // 8
    rec = line_receivers(nrec, n // 2, lo, hi - lo)
    return dict(nx=n, ny=n, c_map=c, c_ref=1.0, source=src, receivers=rec, steps=steps,
                patch=(x0, x0, nxp, nxp), lattice=5, collision="mrt",
                s=[1.0, 1.0, 1.0, 2.0, 2.0], tau=0.5, sponge_width=max(2, int(round(40 * s))),
                sponge_sigma_max=0.1, block=(b0, b0, bw, bw))


def refined_nested_workload(n=2048, nrec=256, steps=4000):
    """The grid-refinement workload with a second, nested patch (ratio 4 to the coarse grid,
    "multiples of 2", Sec. 4): the central half of the first patch's fine grid, inside the
    slow block, refined by 2 again.  The nested patch is given in the first fine grid's node
    coordinates."""
    wl = refined_block_workload(n, nrec, steps)
    nxf = 2 * wl["patch"][2] + 1
    q = (nxf - 1) // 4
    wl["patches"] = [wl["patch"], (q, q, 2 * q, 2 * q)]
    return wl


def layered_workload(n=8192, nrec=512, steps=10000, seed=DEFAULT_SEED + 4, storage="f32"):
    """The 8192^2 layered workload (scaled to n^2 when n differs): a 20-layer model with
    dipping interfaces and 4 normal faults (speeds 1500-5500 m/s, throws 20-200 cells at
    8192 scaled with the grid side), c_ref = 5500 m/s, 10 points per wavelength at
    1500 m/s, Ricker source at (n/2, 80), ``nrec`` receivers on the source row between the
    40-cell sponges, D2Q5 BGK tau = 1/2, ``steps`` steps."""
    f = n / 8192.0
    c = layered_fault_model(n, n, seed, n_layers=20, throw=(20.0 * f, 200.0 * f))
    y = 80
    return dict(nx=n, ny=n, c_map=c, c_ref=SERVED_C_REF, source=(n // 2, y, ricker(steps, SERVED_FC)),
                receivers=line_receivers(nrec, y, 40, n - 80), steps=steps, lattice=5,
                collision="bgk", tau=0.5, sponge_width=40, sponge_sigma_max=0.1, periodic=False,
                storage=storage, w_ref=(4 / 9, 1 / 9, 1 / 36))


# --- served shot stream ---------------------------------------------------------------

SERVED_SIZES = (256, 512, 1024, 2048)
SERVED_C_REF = 5500.0
# 10 points per wavelength at the slowest layer speed (1500 m/s): the D2Q5 lattice
# sound speed there is (1500 / 5500) / sqrt(2) cells per step.
SERVED_FC = (1500.0 / SERVED_C_REF) / math.sqrt(2.0) / 10.0


def served_requests(n_req, seed, sizes=SERVED_SIZES, steps=(2000, 8000), p_bf16=0.5,
                    p_grad=0.25, layers=(4, 12), id0=0):
    """Descriptors of a stream of independent seismic shots (no arrays yet).

    Grid side uniform in ``sizes``, step count uniform integer in ``steps``
    (inclusive), storage BF16 with probability ``p_bf16`` else FP32, an adjoint
    gradient with probability ``p_grad``, and a layered-fault model of
    ``layers`` (inclusive) layers seeded by the request id."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_req):
        out.append(dict(id=id0 + k, n=int(rng.choice(sizes)),
                        nt=int(rng.integers(steps[0], steps[1] + 1)),
                        storage="bf16" if rng.random() < p_bf16 else "f32",
                        grad=bool(rng.random() < p_grad),
                        layers=int(rng.integers(layers[0], layers[1] + 1))))
    return out


def served_shot(desc, nrec=128, sponge=40):
    """Inputs of one served shot: layered-fault model (throws scaled from 20-200
    cells at 8192 to the grid side), Ricker source at (n/2, sponge + 8), ``nrec``
    receivers on the source row between the sponges, D2Q5 BGK tau = 1/2."""
    n = desc["n"]
    f = n / 8192.0
    c = layered_fault_model(n, n, desc["id"], n_layers=desc["layers"],
                            throw=(20.0 * f, 200.0 * f))
    y = sponge + 8
    return dict(c_map=c, nt=desc["nt"], source=(n // 2, y, ricker(desc["nt"], SERVED_FC)),
                receivers=line_receivers(nrec, y, sponge, n - 2 * sponge), lattice=5,
                collision="bgk", tau=0.5, storage=desc["storage"], sponge_width=sponge,
                sponge_sigma_max=0.1, c_ref=SERVED_C_REF, want_gradient=desc["grad"])
