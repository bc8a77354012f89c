"""Seeded synthetic inputs: SU(3) gauge links, complex-Gaussian sources, gauge transforms.

This module holds none of the solver's arithmetic (no staggered operator, no
phases, no CG); it only draws inputs.  Both the CUDA path's tests/benchmark and
the CPU oracle's tests take their inputs from here, so the two sides see the
same FP64 buffers.

The paper (Sec. 3) runs on MILC asqtad 20^3 x 64 gauge ensembles, which are not
available; random fields of the same shape stand in for them:

* link U = reunitarise(exp(i c H)), H traceless Hermitian with N(0,1) entries
  (diagonal H_ii ~ N(0,1); off-diagonal H_ij = a + i b, a, b ~ N(0,1),
  H_ji = conj(H_ij); the trace/3 is removed from the diagonal).  exp is taken
  through the eigendecomposition of H.  Reunitarisation: Gram-Schmidt on rows 0
  and 1, row 2 = conj(row0 x row1), so det U = 1 to rounding.  c sets the
  roughness (0 gives unit links).
* source: re, im iid N(0,1) per colour component.

Layouts are those of the C ABI: links (4, V, 3, 3) complex128 with V in
lexicographic order (x fastest); checkerboard vectors (V/2, 3) complex128.
Random draws use numpy's PCG64 with the seed given; links are drawn in a fixed
order (direction-major, then site) in chunks, so the result does not depend on
the chunk size.
"""
from __future__ import annotations

import numpy as np

_CHUNK = 1 << 20


def volume(dims) -> int:
    return int(np.prod(np.asarray(dims, dtype=np.int64)))


def _hermitian_from_normals(z: np.ndarray) -> np.ndarray:
    """(n, 9) normals -> (n, 3, 3) traceless Hermitian matrices."""
    n = z.shape[0]
    H = np.zeros((n, 3, 3), np.complex128)
    H[:, 0, 0] = z[:, 0]
    H[:, 1, 1] = z[:, 1]
    H[:, 2, 2] = z[:, 2]
    for k, (i, j) in enumerate(((0, 1), (0, 2), (1, 2))):
        h = z[:, 3 + 2 * k] + 1j * z[:, 4 + 2 * k]
        H[:, i, j] = h
        H[:, j, i] = np.conj(h)
    tr = (H[:, 0, 0] + H[:, 1, 1] + H[:, 2, 2]) / 3.0
    for i in range(3):
        H[:, i, i] -= tr
    return H


def reunitarise(U: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on rows 0, 1; row 2 = conj(row0 x row1)."""
    U = np.array(U, dtype=np.complex128, copy=True)
    r0 = U[..., 0, :]
    r0 /= np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 -= np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 /= np.linalg.norm(r1, axis=-1, keepdims=True)
    U[..., 0, :] = r0
    U[..., 1, :] = r1
    U[..., 2, :] = np.conj(np.cross(r0, r1))
    return U


def su3_matrices(rng: np.random.Generator, n: int, c: float) -> np.ndarray:
    """n matrices reunitarise(exp(i c H)), drawn in chunks from rng."""
    out = np.empty((n, 3, 3), np.complex128)
    for s in range(0, n, _CHUNK):
        m = min(_CHUNK, n - s)
        z = rng.standard_normal((m, 9))
        if c == 0.0:
            out[s:s + m] = np.eye(3)
            continue
        H = _hermitian_from_normals(z)
        w, Q = np.linalg.eigh(H)
        E = np.exp(1j * c * w)
        U = np.einsum("nij,nj,nkj->nik", Q, E, np.conj(Q))
        out[s:s + m] = reunitarise(U)
    return out


def random_links(dims, c: float, seed: int) -> np.ndarray:
    """Gauge field (4, V, 3, 3) complex128 of reunitarised exp(i c H) links."""
    V = volume(dims)
    rng = np.random.Generator(np.random.PCG64(seed))
    return su3_matrices(rng, 4 * V, c).reshape(4, V, 3, 3)


def _reunitarise_torch(U):
    """reunitarise() on a torch tensor (..., 3, 3)."""
    import torch
    r0 = U[..., 0, :]
    r0 = r0 / torch.linalg.vector_norm(r0, dim=-1, keepdim=True)
    r1 = U[..., 1, :]
    r1 = r1 - torch.sum(torch.conj(r0) * r1, dim=-1, keepdim=True) * r0
    r1 = r1 / torch.linalg.vector_norm(r1, dim=-1, keepdim=True)
    r2 = torch.conj(torch.linalg.cross(r0, r1, dim=-1))
    return torch.stack((r0, r1, r2), dim=-2)


def random_links_device(dims, c: float, seed: int, device="cuda"):
    """random_links() evaluated with torch on `device`, for lattices where the
    numpy eigendecomposition is slow (48^3 x 96 has 42.5 M links).

    The normals are the same draws in the same order and chunks as
    random_links(); exp(i c H) is taken by torch.linalg.matrix_exp instead of
    the eigendecomposition, so the two agree to rounding.  Returns a
    (4, V, 3, 3) complex128 tensor on `device`.
    """
    import torch
    V = volume(dims)
    n = 4 * V
    rng = np.random.Generator(np.random.PCG64(seed))
    out = torch.empty((n, 3, 3), dtype=torch.complex128, device=device)
    for s in range(0, n, _CHUNK):
        m = min(_CHUNK, n - s)
        z = rng.standard_normal((m, 9))
        if c == 0.0:
            out[s:s + m] = torch.eye(3, dtype=torch.complex128, device=device)
            continue
        H = torch.from_numpy(_hermitian_from_normals(z)).to(device)
        out[s:s + m] = _reunitarise_torch(torch.linalg.matrix_exp((1j * c) * H))
    return out.reshape(4, V, 3, 3)


def unit_links(dims) -> np.ndarray:
    V = volume(dims)
    U = np.zeros((4, V, 3, 3), np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def gaussian_vector(n_sites: int, seed: int) -> np.ndarray:
    """(n_sites, 3) complex128 with re, im iid N(0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal((n_sites, 3, 2))
    return z[..., 0] + 1j * z[..., 1]


def gauge_transform(dims, seed: int, c: float = 1.0) -> np.ndarray:
    """A random SU(3) matrix per site, shape (V, 3, 3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return su3_matrices(rng, volume(dims), c)


def seed_for(config: int, stream: int) -> int:
    """Seed convention: 1000 * config + stream id."""
    return 1000 * int(config) + int(stream)
