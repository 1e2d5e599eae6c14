"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generators only -- none of the method's arithmetic.
Both the CPU oracle and the CUDA path read the bytes it produces, so a test
generates an input once and hands the same array to both sides.

The paper measures on one octave of Perlin noise and on the AT-complex
dataset (Experiments section); neither is available here, so seeded sums of
isotropic Gaussians, i.i.d. white noise, thresholded Gaussian sums and a
randomly thinned Kuhn tetrahedral mesh stand in for them.

Recipe (all parameters from ``numpy.random.default_rng(seed)``, drawn in the
order centres, sigmas, amplitudes, then noise):
  * Gaussian sum: ``sum_i A_i exp(-|p-c_i|^2 / (2 sigma_i^2))`` over grid
    points p = (x, y, z); centres uniform in [0, n) per axis; evaluated in
    float64 as a separable product per Gaussian, summed in generation order,
    rounded once to float32.
  * white noise: ``rng.random(n, dtype=float32)`` (multiples of 2^-24, so a
    512^3 field has many exact ties).
  * feature mask: uint8 (Gaussian sum > threshold).
  * Kuhn mesh: every cube split into the 6 tetrahedra 0 -> e_a -> e_a+e_b ->
    (1,1,1); a random fraction of tetrahedra deleted; vertex ids permuted;
    symmetric, row-sorted, de-duplicated int32 CSR of the tetrahedra's edges.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import torch

# ----------------------------------------------------------------------------
# fields


def gaussian_params(dims, count, sigma_range, seed, amp_range=(-1.0, 1.0), rng=None):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed) if rng is None else rng
    centres = rng.uniform(0.0, 1.0, size=(count, 3)) * np.array([nx, ny, nz], np.float64)
    sigmas = rng.uniform(sigma_range[0], sigma_range[1], size=count)
    amps = rng.uniform(amp_range[0], amp_range[1], size=count)
    return centres, sigmas, amps, rng


def gaussian_sum(dims, centres, sigmas, amps, device="cpu", noise=None) -> torch.Tensor:
    """float32 tensor of shape (nz, ny, nx) (x fastest in memory)."""
    nx, ny, nz = dims
    dev = torch.device(device)
    acc = torch.zeros((nz, ny, nx), dtype=torch.float64, device=dev)
    xs = torch.arange(nx, dtype=torch.float64, device=dev)
    ys = torch.arange(ny, dtype=torch.float64, device=dev)
    zs = torch.arange(nz, dtype=torch.float64, device=dev)
    for (cx, cy, cz), s, a in zip(centres, sigmas, amps):
        k = -1.0 / (2.0 * float(s) * float(s))
        ex = torch.exp(k * (xs - float(cx)) ** 2)
        ey = torch.exp(k * (ys - float(cy)) ** 2)
        ez = torch.exp(k * (zs - float(cz)) ** 2)
        yz = (float(a) * ez)[:, None] * ey[None, :]
        acc.addcmul_(yz[:, :, None], ex[None, None, :])
    if noise is not None:
        acc += torch.as_tensor(noise, dtype=torch.float64, device=dev).view(nz, ny, nx)
    return acc.to(torch.float32)


def smooth_field(dims, count, sigma_range, seed, device="cpu", noise_amp=0.0):
    centres, sigmas, amps, rng = gaussian_params(dims, count, sigma_range, seed)
    noise = None
    if noise_amp > 0.0:
        noise = rng.uniform(0.0, noise_amp, size=int(np.prod(dims)))
    return gaussian_sum(dims, centres, sigmas, amps, device=device, noise=noise)


def white_noise(dims, seed, device="cpu") -> torch.Tensor:
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    a = rng.random(nx * ny * nz, dtype=np.float32)
    return torch.from_numpy(a).view(nz, ny, nx).to(device)


def feature_mask(dims, count, sigma_range, threshold, seed, device="cpu") -> torch.Tensor:
    f = smooth_field(dims, count, sigma_range, seed, device=device)
    return (f > threshold).to(torch.uint8)


# Named workloads: a 64^3 field of 8 Gaussians (sigma 4..12) plus U[0,1e-3]
# noise; 512^3 fields, smooth (64 Gaussians, sigma 32..96) or white noise;
# a 1024^3 feature mask (256 Gaussians, sigma 64..192, threshold 0.3).


def field_small(device="cpu", edge=64, seed=0):
    return smooth_field((edge,) * 3, 8, (4.0, 12.0), seed, device=device, noise_amp=1e-3)


def field_smooth(edge=512, seed=1, device="cpu"):
    s = edge / 512.0 * 64.0
    return smooth_field((edge,) * 3, 64, (0.5 * s, 1.5 * s), seed, device=device)


def field_noise(edge=512, seed=1, device="cpu"):
    return white_noise((edge,) * 3, seed, device=device)


def mask_blobs(edge=1024, seed=2, device="cpu", threshold=0.3):
    s = edge / 1024.0 * 128.0
    return feature_mask((edge,) * 3, 256, (0.5 * s, 1.5 * s), threshold, seed, device=device)


def mask_top(edge=1024, seed=2, top=0.1, device="cpu", sample=1 << 22):
    """The feature mask of the paper's density sweep: the voxels holding the
    top `top` fraction of the blob field's values (the mask_blobs field).
    The threshold is the (1 - top) quantile of a seeded sample of 2^22
    voxels, so the masked fraction is `top` to within about a thousandth."""
    s = edge / 1024.0 * 128.0
    f = smooth_field((edge,) * 3, 256, (0.5 * s, 1.5 * s), seed, device=device).reshape(-1)
    g = torch.Generator(device=f.device).manual_seed(seed)
    idx = torch.randint(0, f.numel(), (min(sample, f.numel()),), device=f.device, generator=g)
    thr = torch.quantile(f[idx].double(), 1.0 - top).item()
    return (f > thr).to(torch.uint8).reshape((edge,) * 3)


# ----------------------------------------------------------------------------
# tetrahedral mesh

KUHN_PERMS = list(itertools.permutations(range(3)))


def kuhn_tets(edge: int, device="cpu") -> torch.Tensor:
    """(6 * (edge-1)^3, 4) int64 vertex ids of the Kuhn split, grid ids."""
    dev = torch.device(device)
    c = edge - 1
    r = torch.arange(c, device=dev, dtype=torch.int64)
    z, y, x = torch.meshgrid(r, r, r, indexing="ij")
    base = (x + edge * (y + edge * z)).reshape(-1)
    step = [1, edge, edge * edge]
    tets = []
    for p in KUHN_PERMS:
        v1 = base + step[p[0]]
        v2 = v1 + step[p[1]]
        v3 = v2 + step[p[2]]
        tets.append(torch.stack([base, v1, v2, v3], dim=1))
    return torch.stack(tets, dim=1).reshape(-1, 4)


def tet_mesh_csr(edge=256, delete_frac=0.4, seed=3, device="cpu"):
    """Symmetric int32 CSR (row, col) of a thinned, permuted Kuhn mesh."""
    n = edge ** 3
    tets = kuhn_tets(edge, device=device)
    rng = np.random.default_rng(seed)
    keep = rng.random(tets.shape[0], dtype=np.float32) >= np.float32(delete_frac)
    perm = rng.permutation(n)
    dev = tets.device
    tets = tets[torch.from_numpy(keep).to(dev)]
    perm_t = torch.from_numpy(perm.astype(np.int64)).to(dev)
    tets = perm_t[tets]
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    a = torch.cat([tets[:, i] for i, _ in pairs])
    b = torch.cat([tets[:, j] for _, j in pairs])
    del tets
    lo = torch.minimum(a, b)
    hi = torch.maximum(a, b)
    del a, b
    und = torch.unique(lo * n + hi)
    del lo, hi
    u = und // n
    w = und % n
    rows = torch.cat([u, w])
    cols = torch.cat([w, u])
    del und, u, w
    key = torch.sort(rows * n + cols).values
    rows = key // n
    cols = (key % n).to(torch.int32)
    counts = torch.bincount(rows, minlength=n)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(counts, 0)
    return row_ptr.to(torch.int32), cols


# ----------------------------------------------------------------------------
# batched and served workloads


def batch_dims(seed: int):
    """Per-instance grid shape: each axis edge round(exp(U[ln 16, ln 256]))."""
    rng = np.random.default_rng(seed)
    e = np.rint(np.exp(rng.uniform(math.log(16.0), math.log(256.0), size=3))).astype(int)
    return (int(e[0]), int(e[1]), int(e[2])), rng


def batch_instance(seed: int, device="cpu"):
    """One batched instance: anisotropic grid, 8 Gaussians, sigma scaled by
    the geometric-mean edge / 64."""
    dims, rng = batch_dims(seed)
    g = (dims[0] * dims[1] * dims[2]) ** (1.0 / 3.0) / 64.0
    centres, sigmas, amps, _ = gaussian_params(dims, 8, (4.0 * g, 12.0 * g), None, rng=rng)
    return dims, gaussian_sum(dims, centres, sigmas, amps, device=device)


def serve_request(seed: int):
    """A served job: 70 % Morse-Smale segmentation on a cube of edge
    log-uniform in [32, 512], 30 % mask CC on a cube of edge log-uniform in
    [64, 768].  Returns (kind, edge, rng) -- fields are drawn by the caller
    with ``serve_field``."""
    rng = np.random.default_rng(seed)
    if rng.random() < 0.7:
        edge = int(round(math.exp(rng.uniform(math.log(32), math.log(512)))))
        return "segment", edge, rng
    edge = int(round(math.exp(rng.uniform(math.log(64), math.log(768)))))
    return "cc", edge, rng


def serve_field(kind: str, edge: int, rng, device="cpu"):
    dims = (edge,) * 3
    g = edge / 64.0
    centres, sigmas, amps, _ = gaussian_params(dims, 8, (4.0 * g, 12.0 * g), None, rng=rng)
    f = gaussian_sum(dims, centres, sigmas, amps, device=device)
    if kind == "cc":
        return (f > 0.3).to(torch.uint8)
    return f


def serve_job(seed: int, device="cpu"):
    """A served request with its own seeded input: (kind, dims, tensor) with
    the kind and cube edge of ``serve_request(seed)`` and, from the same
    generator, 8 Gaussians (sigma 4..12 scaled by edge / 64) evaluated in
    float32 as one (nz*ny x 8) @ (8 x nx) product of the separable factors
    -- a single write pass, so that a request's input can be made just
    before it is submitted.  CC requests get the mask (field > 0.3)."""
    kind, edge, rng = serve_request(seed)
    dims = (edge,) * 3
    g = edge / 64.0
    centres, sigmas, amps, _ = gaussian_params(dims, 8, (4.0 * g, 12.0 * g), None, rng=rng)
    dev = torch.device(device)
    r = torch.arange(edge, dtype=torch.float32, device=dev)
    c = torch.as_tensor(centres, dtype=torch.float32, device=dev)
    k = torch.as_tensor(-1.0 / (2.0 * sigmas * sigmas), dtype=torch.float32, device=dev)[:, None]
    a = torch.as_tensor(amps, dtype=torch.float32, device=dev)
    ex = torch.exp(k * (r[None, :] - c[:, 0:1]) ** 2)
    ey = torch.exp(k * (r[None, :] - c[:, 1:2]) ** 2)
    ez = torch.exp(k * (r[None, :] - c[:, 2:3]) ** 2)
    m = (a[:, None, None] * ez[:, :, None] * ey[:, None, :]).reshape(len(amps), -1)
    f = (m.t() @ ex).reshape(-1)
    if kind == "cc":
        return kind, dims, (f > 0.3).to(torch.uint8)
    return kind, dims, f
