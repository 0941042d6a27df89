"""3D linear elasticity on the unit cube with trilinear (Q1) or triquadratic
(Q2) hexahedra.

Problem inputs for the blocked smoothed-aggregation AMG reuse phase: the
mesh, the 24x24 element stiffness, the blocked COO value stream (one 3x3 block
per pair of element nodes, 64 per element, duplicates left for the assembler
to sum), the consistent body-force load and the seeded perturbations and
right-hand sides.  The paper's harnesses are not available, so this is our own
generator for the workloads the paper measures: Q1 hexahedral 3D elasticity,
block size 3 (Sec. 4.1), assembled through blocked COO (Sec. 3.4, Sec. 5).

Conventions (all fixed here and used by every consumer):
  * ``ne`` elements per direction of side ``h = 1 / ne``, element order
    ``p`` (1: Q1, 8 nodes; 2: Q2, 27 nodes), ``m = p*ne + 1`` nodes per
    direction at spacing ``h / p``; node ``n = ix + m*iy + m*m*iz`` at
    ``(ix, iy, iz) * h / p``.
  * element ``e = ex + ne*ey + ne*ne*ez``; local node
    ``a = bx + (p+1)*by + (p+1)^2*bz`` with ``bx, by, bz`` in ``0..p``.
  * dof ``3*n + c`` for displacement component ``c``.
  * Dirichlet: every node with ``ix == 0`` is clamped in all 3 components.
    Element blocks touching a clamped node are zero, and one extra identity
    block per clamped node is appended to the stream, so the assembled
    operator has zero rows/columns there and an identity diagonal block while
    every structural block stays in the pattern.
  * Element stiffness ``K_e = (E_e * h) * K_ref(nu)`` where ``K_ref`` is the
    stiffness of the unit cube with E = 1 (stiffness scales with E and, in
    3D, linearly with the element size h).  Q1 uses 2x2x2 Gauss points and
    Q2 3x3x3, exact for both stiffnesses on a cube.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch


@dataclasses.dataclass(frozen=True)
class Mesh:
    ne: int
    order: int = 1

    @property
    def m(self) -> int:
        return self.order * self.ne + 1

    @property
    def h(self) -> float:
        """Element side."""
        return 1.0 / self.ne

    @property
    def nodes_per_element(self) -> int:
        return (self.order + 1) ** 3

    @property
    def n_nodes(self) -> int:
        return self.m ** 3

    @property
    def n_dofs(self) -> int:
        return 3 * self.n_nodes

    @property
    def n_el(self) -> int:
        return self.ne ** 3

    @property
    def grid(self) -> tuple[int, int, int]:
        return (self.m, self.m, self.m)

    def node_ijk(self) -> np.ndarray:
        n = np.arange(self.n_nodes, dtype=np.int64)
        m = self.m
        return np.stack([n % m, (n // m) % m, n // (m * m)], axis=1)

    def coords(self) -> np.ndarray:
        return self.node_ijk().astype(np.float64) * (self.h / self.order)

    def dirichlet(self) -> np.ndarray:
        return (self.node_ijk()[:, 0] == 0).astype(np.uint8)

    def connectivity(self) -> np.ndarray:
        ne, m = self.ne, self.m
        e = np.arange(self.n_el, dtype=np.int64)
        ex, ey, ez = e % ne, (e // ne) % ne, e // (ne * ne)
        p = self.order
        base = p * (ex + m * ey + m * m * ez)
        a = np.arange((p + 1) ** 3)
        off = (a % (p + 1)) + m * ((a // (p + 1)) % (p + 1)) + m * m * (a // (p + 1) ** 2)
        return base[:, None] + off[None, :]

    def element_centroids(self) -> np.ndarray:
        ne = self.ne
        e = np.arange(self.n_el, dtype=np.int64)
        ijk = np.stack([e % ne, (e // ne) % ne, e // (ne * ne)], axis=1)
        return (ijk.astype(np.float64) + 0.5) * self.h


def gauss_rule(order: int) -> tuple[np.ndarray, np.ndarray]:
    """Gauss-Legendre points and weights on [0, 1]."""
    if order == 2:
        s = 0.5 / np.sqrt(3.0)
        return np.array([0.5 - s, 0.5 + s]), np.array([0.5, 0.5])
    if order == 3:
        s = 0.5 * np.sqrt(0.6)
        return np.array([0.5 - s, 0.5, 0.5 + s]), np.array([5.0, 8.0, 5.0]) / 18.0
    raise ValueError("order must be 2 or 3")


def lame(E: float, nu: float) -> tuple[float, float]:
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def lagrange_1d(degree: int, t: float) -> tuple[np.ndarray, np.ndarray]:
    """Values and derivatives of the 1-D Lagrange basis on [0, 1] with
    equispaced nodes (degree 1: 0, 1; degree 2: 0, 1/2, 1)."""
    if degree == 1:
        return np.array([1.0 - t, t]), np.array([-1.0, 1.0])
    if degree == 2:
        return (np.array([(1.0 - t) * (1.0 - 2.0 * t), 4.0 * t * (1.0 - t), t * (2.0 * t - 1.0)]),
                np.array([4.0 * t - 3.0, 4.0 - 8.0 * t, 4.0 * t - 1.0]))
    raise ValueError("degree must be 1 or 2")


def element_stiffness_q(E: float, nu: float, h: float, degree: int, order: int) -> np.ndarray:
    """Isotropic Q1 / Q2 stiffness of a cube of side h with ``order`` Gauss
    points per direction; dofs ordered 3*a + c, a = bx + (p+1) by + (p+1)^2 bz."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[[0, 1, 2], [0, 1, 2]] += 2.0 * mu
    D[[3, 4, 5], [3, 4, 5]] = mu
    pts, wts = gauss_rule(order)
    q = degree + 1
    nn = q ** 3
    idx = np.array([[a % q, (a // q) % q, a // (q * q)] for a in range(nn)])
    K = np.zeros((3 * nn, 3 * nn))
    for i, xi in enumerate(pts):
        for j, eta in enumerate(pts):
            for k, zeta in enumerate(pts):
                (fx, dx), (fy, dy), (fz, dz) = (lagrange_1d(degree, t) for t in (xi, eta, zeta))
                grad = np.stack([dx[idx[:, 0]] * fy[idx[:, 1]] * fz[idx[:, 2]],
                                 fx[idx[:, 0]] * dy[idx[:, 1]] * fz[idx[:, 2]],
                                 fx[idx[:, 0]] * fy[idx[:, 1]] * dz[idx[:, 2]]], axis=1) / h
                B = np.zeros((6, 3 * nn))
                for a in range(nn):
                    gx, gy, gz = grad[a]
                    c = 3 * a
                    B[0, c] = gx
                    B[1, c + 1] = gy
                    B[2, c + 2] = gz
                    B[3, c], B[3, c + 1] = gy, gx
                    B[4, c + 1], B[4, c + 2] = gz, gy
                    B[5, c], B[5, c + 2] = gz, gx
                w = wts[i] * wts[j] * wts[k] * h ** 3
                K += w * (B.T @ D @ B)
    return K


def element_stiffness(E: float, nu: float, h: float = 1.0, order: int = 2) -> np.ndarray:
    """24x24 isotropic Q1 stiffness of a cube of side h, dofs ordered 3*a + c."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[[0, 1, 2], [0, 1, 2]] += 2.0 * mu
    D[[3, 4, 5], [3, 4, 5]] = mu
    pts, wts = gauss_rule(order)
    bits = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)])
    K = np.zeros((24, 24))
    for i, xi in enumerate(pts):
        for j, eta in enumerate(pts):
            for k, zeta in enumerate(pts):
                q = np.array([xi, eta, zeta])
                f = np.where(bits == 1, q, 1.0 - q)          # 1-D factors per node
                df = np.where(bits == 1, 1.0, -1.0)          # their derivatives
                grad = np.stack([df[:, 0] * f[:, 1] * f[:, 2],
                                 f[:, 0] * df[:, 1] * f[:, 2],
                                 f[:, 0] * f[:, 1] * df[:, 2]], axis=1) / h
                B = np.zeros((6, 24))
                for a in range(8):
                    gx, gy, gz = grad[a]
                    c = 3 * a
                    B[0, c] = gx
                    B[1, c + 1] = gy
                    B[2, c + 2] = gz
                    B[3, c], B[3, c + 1] = gy, gx
                    B[4, c + 1], B[4, c + 2] = gz, gy
                    B[5, c], B[5, c + 2] = gz, gx
                w = wts[i] * wts[j] * wts[k] * h ** 3
                K += w * (B.T @ D @ B)
    return K


def reference_blocks(nu: float, degree: int = 1) -> np.ndarray:
    """K_ref(nu) cut into its nn^2 3x3 blocks (nn = 8 or 27 nodes), ordered
    (a, b) -> nn*a + b."""
    if degree == 1:
        K = element_stiffness(1.0, nu, 1.0, 2)
    else:
        K = element_stiffness_q(1.0, nu, 1.0, degree, degree + 1)
    nn = (degree + 1) ** 3
    return K.reshape(nn, 3, nn, 3).transpose(0, 2, 1, 3).reshape(nn * nn, 3, 3).copy()


def element_scale(mesh: Mesh, E_el: np.ndarray | None = None,
                  delta: np.ndarray | None = None) -> np.ndarray:
    """Per-element factor c_e = h * E_e * (1 + delta_e)."""
    E = np.ones(mesh.n_el) if E_el is None else np.asarray(E_el, dtype=np.float64)
    c = mesh.h * E
    if delta is not None:
        c = c * (1.0 + np.asarray(delta, dtype=np.float64))
    return c


@dataclasses.dataclass
class CooStream:
    """Blocked COO stream: block coordinates and row-major 3x3 value blocks."""
    bi: torch.Tensor      # int32 (n_coo,)
    bj: torch.Tensor      # int32 (n_coo,)
    vals: torch.Tensor    # float64 (n_coo, 3, 3)

    @property
    def n(self) -> int:
        return int(self.bi.shape[0])


def coo_indices(mesh: Mesh, device="cpu") -> tuple[torch.Tensor, torch.Tensor]:
    conn = torch.as_tensor(mesh.connectivity(), device=device)
    n_el, nn = conn.shape
    bi = conn[:, :, None].expand(n_el, nn, nn).reshape(-1)
    bj = conn[:, None, :].expand(n_el, nn, nn).reshape(-1)
    dn = torch.as_tensor(np.nonzero(mesh.dirichlet())[0], device=device)
    bi = torch.cat([bi, dn]).to(torch.int32)
    bj = torch.cat([bj, dn]).to(torch.int32)
    return bi, bj


def coo_values(mesh: Mesh, nu: float, scale: np.ndarray, device="cpu",
               out: torch.Tensor | None = None) -> torch.Tensor:
    """Value stream (n_coo, 3, 3) float64 matching :func:`coo_indices`.

    Element values are ``scale[e] * K_ref`` (one IEEE multiply, identical on
    host and device); blocks touching a clamped node are exact zeros; the
    trailing clamped-node blocks are identities.
    """
    kb = torch.as_tensor(reference_blocks(nu, mesh.order), device=device)
    s = torch.as_tensor(np.asarray(scale, dtype=np.float64), device=device)
    conn = torch.as_tensor(mesh.connectivity(), device=device)
    dirn = torch.as_tensor(mesh.dirichlet().astype(bool), device=device)
    n_el, nn = conn.shape
    nb = nn * nn
    n_dir = int(mesh.dirichlet().sum())
    n_coo = nb * n_el + n_dir
    if out is None:
        out = torch.empty((n_coo, 3, 3), dtype=torch.float64, device=device)
    el = out[: nb * n_el].view(n_el, nb, 3, 3)
    torch.mul(s[:, None, None, None], kb[None], out=el)
    dn = dirn[conn]                                             # (n_el, nn)
    touch = (dn[:, :, None] | dn[:, None, :]).reshape(n_el, nb)  # (n_el, nn^2)
    el.masked_fill_(touch[:, :, None, None], 0.0)
    out[nb * n_el:] = torch.eye(3, dtype=torch.float64, device=device)
    return out


def coo_stream(mesh: Mesh, nu: float, scale: np.ndarray, device="cpu") -> CooStream:
    bi, bj = coo_indices(mesh, device)
    return CooStream(bi, bj, coo_values(mesh, nu, scale, device))


def body_force(mesh: Mesh) -> np.ndarray:
    """Consistent load of the unit body force f = (0, 0, -1); zero on clamped dofs.

    Each element node receives minus the integral of its shape function over
    the element in z: h^3/8 for Q1; for Q2 the product of the 1-D quadratic
    weights (1/6, 2/3, 1/6) times h^3.
    """
    f = np.zeros(mesh.n_nodes)
    if mesh.order == 1:
        w = np.full(8, 1.0 / 8.0)
    else:
        w1 = np.array([1.0, 4.0, 1.0]) / 6.0
        w = np.array([w1[a % 3] * w1[(a // 3) % 3] * w1[a // 9] for a in range(27)])
    conn = mesh.connectivity()
    np.add.at(f, conn.reshape(-1), np.tile(-(mesh.h ** 3) * w, conn.shape[0]))
    b = np.zeros((mesh.n_nodes, 3))
    b[:, 2] = f
    b[mesh.dirichlet().astype(bool)] = 0.0
    return b.reshape(-1)


def perturbation(n_el: int, seed: int, amplitude: float = 0.01) -> np.ndarray:
    """Per-element stiffness perturbation delta_e ~ U[-amplitude, amplitude]."""
    return np.random.default_rng(seed).uniform(-amplitude, amplitude, n_el)


def gaussian_rhs(mesh: Mesh, seed: int) -> np.ndarray:
    """N(0, 1) right-hand side with clamped dofs zeroed."""
    b = np.random.default_rng(seed).standard_normal(mesh.n_dofs).reshape(-1, 3)
    b[mesh.dirichlet().astype(bool)] = 0.0
    return b.reshape(-1)


def inclusion_moduli(mesh: Mesh, seed: int) -> np.ndarray:
    """Young's modulus per element: 1 outside, 10^U[-2,2] inside random spheres.

    4..16 spheres with centres U[0,1]^3 and radii U[0.05, 0.15]; an element
    whose centroid lies in several spheres takes the last one's modulus.
    """
    rng = np.random.default_rng(seed)
    k = int(rng.integers(4, 17))
    centres = rng.uniform(0.0, 1.0, (k, 3))
    radii = rng.uniform(0.05, 0.15, k)
    moduli = 10.0 ** rng.uniform(-2.0, 2.0, k)
    E = np.ones(mesh.n_el)
    xc = mesh.element_centroids()  # element geometry: the same for Q1 and Q2
    for c, r, Ek in zip(centres, radii, moduli):
        inside = np.sum((xc - c) ** 2, axis=1) <= r * r
        E[inside] = Ek
    return E


def batch_problems(seed: int = 7, count: int = 32) -> list[tuple[int, float]]:
    """(elements per direction, Poisson ratio) for a batch of uneven problems."""
    rng = np.random.default_rng(seed)
    ne = rng.integers(16, 41, count)
    nu = rng.uniform(0.2, 0.45, count)
    return [(int(a), float(b)) for a, b in zip(ne, nu)]
