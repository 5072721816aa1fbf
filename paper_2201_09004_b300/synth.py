"""Seeded synthetic inputs: gauge links, fat/long links and sources.

This module is input generation only. It holds none of the operator or solver
arithmetic; both the CUDA path and the FP64 CPU oracle read the arrays it
returns. Everything is derived from a counter-based generator, so a field is a
pure function of (seed, field id, site, direction, component) and does not
depend on the device it is generated on or on the order of generation.

Canonical layouts (complex128, C order):
  gauge   [mu][t][z][y][x][3][3]   link U_mu(x): parallel transporter x -> x+mu
  spinor  [t][z][y][x][4][3]       Wilson field, [spin][colour]
  colour  [t][z][y][x][3]          staggered field
Site order is lexicographic, i = x + Lx*(y + Ly*(z + Lz*t)); dims = (Lx, Ly, Lz, Lt).

Generator recipe (the paper fixes none of this; the lattice shapes follow the
ensembles of Table 1):
  * thin links  U = exp(i*eps*H), H = sum_a h_a lambda_a / sqrt(2), h_a ~ N(0,1),
    lambda_a the Gell-Mann matrices. At eps = 0.3 the average plaquette is ~0.61.
  * fat links   V = s*(U' + 0.1*Z), U' a fresh thin link, Z iid complex Gaussian,
    s chosen per link so that ||V||_F = sqrt(3) (non-unitary, "near unity").
  * long links  W_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu) of a separate thin field
    (unsigned; the antiperiodic sign belongs to the operator, not the link).
  * Z2 complex noise: each component (+-1 +- i)/sqrt(2), independent bits.
"""
from __future__ import annotations

import math

import torch

# SplitMix64 constants (Steele, Lea, Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014), written as signed int64 two's-complement values.
_GOLDEN = 0x9E3779B97F4A7C15 - (1 << 64)
_MIX1 = 0xBF58476D1CE4E5B9 - (1 << 64)
_MIX2 = 0x94D049BB133111EB - (1 << 64)

# field ids keep the streams of different fields apart
FID_THIN = 1
FID_FAT_U = 2
FID_FAT_Z = 3
FID_LONG_U = 4
FID_SOURCE = 5
FID_GAUGE_TRANSFORM = 6
FID_POINT = 7


def _srl(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 holding uint64 bit patterns."""
    return torch.bitwise_and(torch.bitwise_right_shift(z, k), (1 << (64 - k)) - 1)


def splitmix64(x: torch.Tensor) -> torch.Tensor:
    """SplitMix64 finaliser on int64 tensors (wrapping arithmetic mod 2^64)."""
    z = x + _GOLDEN
    z = torch.bitwise_xor(z, _srl(z, 30)) * _MIX1
    z = torch.bitwise_xor(z, _srl(z, 27)) * _MIX2
    return torch.bitwise_xor(z, _srl(z, 31))


def _key(seed: int, fid: int) -> int:
    k = splitmix64(torch.tensor([(seed * 1000003 + fid) & ((1 << 63) - 1)], dtype=torch.int64))
    return int(k.item())


def random_bits(seed: int, fid: int, counter: torch.Tensor) -> torch.Tensor:
    """64 random bits per counter value: splitmix64(key + splitmix64(counter))."""
    return splitmix64(splitmix64(counter) + _key(seed, fid))


def uniform01(bits: torch.Tensor) -> torch.Tensor:
    """Uniform in (0, 1]: top 53 bits, offset by one ulp so log() is finite."""
    return (_srl(bits, 11) + 1).to(torch.float64) * (2.0 ** -53)


def normals(seed: int, fid: int, counter: torch.Tensor) -> torch.Tensor:
    """Two standard normals per counter (Box-Muller); returns shape counter.shape + (2,)."""
    u1 = uniform01(random_bits(seed, fid, counter * 2))
    u2 = uniform01(random_bits(seed, fid, counter * 2 + 1))
    r = torch.sqrt(-2.0 * torch.log(u1))
    th = 2.0 * math.pi * u2
    return torch.stack([r * torch.cos(th), r * torch.sin(th)], dim=-1)


def volume(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def _shape4(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def gell_mann(device="cpu") -> torch.Tensor:
    """The eight Gell-Mann matrices, tr(l_a l_b) = 2 delta_ab; shape (8, 3, 3)."""
    g = torch.zeros(8, 3, 3, dtype=torch.complex128)
    g[0, 0, 1] = g[0, 1, 0] = 1
    g[1, 0, 1] = -1j
    g[1, 1, 0] = 1j
    g[2, 0, 0] = 1
    g[2, 1, 1] = -1
    g[3, 0, 2] = g[3, 2, 0] = 1
    g[4, 0, 2] = -1j
    g[4, 2, 0] = 1j
    g[5, 1, 2] = g[5, 2, 1] = 1
    g[6, 1, 2] = -1j
    g[6, 2, 1] = 1j
    g[7, 0, 0] = g[7, 1, 1] = 1 / math.sqrt(3)
    g[7, 2, 2] = -2 / math.sqrt(3)
    return g.to(device)


def _site_mu_counter(dims, mu: int, device) -> torch.Tensor:
    v = volume(dims)
    return (torch.arange(v, dtype=torch.int64, device=device) * 4 + mu)


def _su3_near_unity(dims, seed: int, fid: int, eps: float, mu: int, device) -> torch.Tensor:
    """exp(i eps H) for every site of direction mu; shape (V, 3, 3)."""
    ctr = _site_mu_counter(dims, mu, device)                      # (V,)
    # 8 normals per link: counters ctr*4 + k, k = 0..3, two normals each
    k = torch.arange(4, dtype=torch.int64, device=device)
    h = normals(seed, fid, ctr[:, None] * 4 + k[None, :]).reshape(-1, 8)
    lam = gell_mann(device)
    herm = torch.einsum("va,aij->vij", h.to(torch.complex128), lam) / math.sqrt(2.0)
    return torch.linalg.matrix_exp(1j * eps * herm)


def thin_links(dims, seed: int, eps: float = 0.3, device="cpu", fid: int = FID_THIN) -> torch.Tensor:
    """SU(3) links U_mu(x) = exp(i eps H); shape (4, Lt, Lz, Ly, Lx, 3, 3) complex128."""
    out = torch.empty((4,) + _shape4(dims) + (3, 3), dtype=torch.complex128, device=device)
    for mu in range(4):
        out[mu] = _su3_near_unity(dims, seed, fid, eps, mu, device).reshape(_shape4(dims) + (3, 3))
    return out


def unit_links(dims, device="cpu") -> torch.Tensor:
    """Free field U = 1."""
    out = torch.zeros((4,) + _shape4(dims) + (3, 3), dtype=torch.complex128, device=device)
    out[..., 0, 0] = out[..., 1, 1] = out[..., 2, 2] = 1
    return out


def fat_links(dims, seed: int, eps: float = 0.3, noise: float = 0.1, device="cpu") -> torch.Tensor:
    """Non-unitary fat links V = s (U' + noise Z), ||V||_F = sqrt(3) per link."""
    out = torch.empty((4,) + _shape4(dims) + (3, 3), dtype=torch.complex128, device=device)
    for mu in range(4):
        u = _su3_near_unity(dims, seed, FID_FAT_U, eps, mu, device)
        ctr = _site_mu_counter(dims, mu, device)
        k = torch.arange(9, dtype=torch.int64, device=device)
        z = normals(seed, FID_FAT_Z, ctr[:, None] * 9 + k[None, :])       # (V, 9, 2)
        zc = torch.complex(z[..., 0], z[..., 1]).reshape(-1, 3, 3) / math.sqrt(2.0)
        v = u + noise * zc
        nrm = torch.linalg.matrix_norm(v, ord="fro")
        v = v * (math.sqrt(3.0) / nrm)[:, None, None]
        out[mu] = v.reshape(_shape4(dims) + (3, 3))
    return out


def long_links(dims, seed: int, eps: float = 0.3, device="cpu") -> torch.Tensor:
    """W_mu(x) = U_mu(x) U_mu(x+mu) U_mu(x+2mu) of a separate thin field (periodic wrap)."""
    u = thin_links(dims, seed, eps, device=device, fid=FID_LONG_U)
    out = torch.empty_like(u)
    # array axes of (Lt, Lz, Ly, Lx): direction mu=0 (x) is axis 3, mu=3 (t) is axis 0
    for mu in range(4):
        ax = 3 - mu
        u1 = torch.roll(u[mu], shifts=-1, dims=ax)
        u2 = torch.roll(u[mu], shifts=-2, dims=ax)
        out[mu] = u[mu] @ u1 @ u2
    return out


def z2_source(dims, seed: int, ncomp: int = 12, device="cpu", real: bool = False) -> torch.Tensor:
    """Z2 noise: each component (+-1 +- i)/sqrt(2) (or +-1 when real=True).

    Shape (Lt, Lz, Ly, Lx, 4, 3) for ncomp=12, (Lt, Lz, Ly, Lx, 3) for ncomp=3.
    """
    v = volume(dims)
    ctr = torch.arange(v * ncomp, dtype=torch.int64, device=device)
    bits = random_bits(seed, FID_SOURCE, ctr)
    re = 1.0 - 2.0 * torch.bitwise_and(bits, 1).to(torch.float64)
    im = 1.0 - 2.0 * torch.bitwise_and(_srl(bits, 1), 1).to(torch.float64)
    if real:
        s = torch.complex(re, torch.zeros_like(re))
    else:
        s = torch.complex(re, im) / math.sqrt(2.0)
    tail = (4, 3) if ncomp == 12 else (3,)
    return s.reshape(_shape4(dims) + tail)


def gaussian_field(dims, seed: int, ncomp: int = 12, device="cpu", fid: int = FID_SOURCE + 16) -> torch.Tensor:
    """Complex Gaussian field (unit variance per component), for random test vectors."""
    v = volume(dims)
    ctr = torch.arange(v * ncomp, dtype=torch.int64, device=device)
    z = normals(seed, fid, ctr)
    s = torch.complex(z[..., 0], z[..., 1]) / math.sqrt(2.0)
    tail = (4, 3) if ncomp == 12 else (3,)
    return s.reshape(_shape4(dims) + tail)


def point_source(dims, site, spin: int | None, colour: int, device="cpu") -> torch.Tensor:
    """Unit vector at site (x, y, z, t), spin (None for staggered) and colour."""
    x, y, z, t = site
    if spin is None:
        out = torch.zeros(_shape4(dims) + (3,), dtype=torch.complex128, device=device)
        out[t, z, y, x, colour] = 1
    else:
        out = torch.zeros(_shape4(dims) + (4, 3), dtype=torch.complex128, device=device)
        out[t, z, y, x, spin, colour] = 1
    return out


def seeded_site(dims, seed: int):
    """A reproducible site (x, y, z, t) drawn from the counter generator."""
    bits = random_bits(seed, FID_POINT, torch.arange(4, dtype=torch.int64))
    return tuple(int(_srl(bits[i:i + 1], 1).item() % int(dims[i])) for i in range(4))


def random_su3(dims, seed: int, device="cpu") -> torch.Tensor:
    """Random SU(3) matrix per site (a gauge transformation g(x)); shape (Lt,Lz,Ly,Lx,3,3)."""
    u = _su3_near_unity(dims, seed, FID_GAUGE_TRANSFORM, 2.0, 0, device)
    return u.reshape(_shape4(dims) + (3, 3))
