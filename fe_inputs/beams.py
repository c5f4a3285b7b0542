"""Seeded beam meshes, materials and dead loads (inputs only; see package doc)."""
from __future__ import annotations

import dataclasses
import math
from itertools import permutations

import numpy as np

SPACING = 0.01  # m, grid spacing of every workload
H = 0.01        # s, backward-Euler step
ALPHA = 0.1     # Rayleigh mass coefficient
BETA = 0.01     # Rayleigh stiffness coefficient
RHO = 1000.0    # kg/m^3
G_Z = -9.81     # m/s^2

SVK, NEOHOOKE, MOONEY_RIVLIN, COROTATIONAL = 0, 1, 2, 3
TET4, HEX8 = 0, 1


def lame_from_young(E, nu):
    """(E, nu) -> (mu, lambda), the usual isotropic conversion."""
    E = np.asarray(E, dtype=np.float64)
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def _grid_nodes(nx, ny, nz, spacing):
    i, j, k = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    # node index = i + (nx+1)*(j + (ny+1)*k): order nodes by (k, j, i)
    ijk = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    idx = ijk[:, 0] + (nx + 1) * (ijk[:, 1] + (ny + 1) * ijk[:, 2])
    order = np.argsort(idx)
    ijk = ijk[order]
    X = ijk.astype(np.float64) * spacing
    return ijk, X


def _node_id(nx, ny, i, j, k):
    return i + (nx + 1) * (j + (ny + 1) * k)


@dataclasses.dataclass
class TetBeam:
    nx: int
    ny: int
    nz: int
    X: np.ndarray          # [n_nodes, 3] rest positions
    conn: np.ndarray       # [n_elems, 4] int32
    fixed_nodes: np.ndarray  # int32, ascending
    elem_type: int = TET4

    @property
    def n_nodes(self):
        return self.X.shape[0]

    @property
    def n_elems(self):
        return self.conn.shape[0]


@dataclasses.dataclass
class HexBeam(TetBeam):
    elem_type: int = HEX8


def tet_beam(a: int, b: int, c: int, spacing: float = SPACING) -> TetBeam:
    """Beam of a x b x c cubes (ny=a, nz=b, nx=c), 6 Kuhn tets per cube."""
    ny, nz, nx = a, b, c
    ijk, X = _grid_nodes(nx, ny, nz, spacing)
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cubes = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
    corder = np.argsort(cubes[:, 0] + nx * (cubes[:, 1] + ny * cubes[:, 2]))
    cubes = cubes[corder]                        # x fastest, then y, then z
    eye = np.eye(3, dtype=np.int64)
    tets = []
    for perm in permutations((0, 1, 2)):         # lexicographic order
        p0, p1 = perm[0], perm[1]
        offs = [np.zeros(3, np.int64), eye[p0], eye[p0] + eye[p1], np.ones(3, np.int64)]
        verts = [cubes + o for o in offs]
        ids = [_node_id(nx, ny, v[:, 0], v[:, 1], v[:, 2]) for v in verts]
        tets.append(np.stack(ids, axis=1))
    conn = np.stack(tets, axis=1).reshape(-1, 4)  # cube-major, permutation-minor
    # orientation: swap the last two vertices where the signed volume is negative
    d = X[conn[:, 1:]] - X[conn[:, [0]]]
    vol6 = np.einsum("ei,ei->e", d[:, 0], np.cross(d[:, 1], d[:, 2]))
    neg = vol6 < 0
    conn[neg, 2], conn[neg, 3] = conn[neg, 3].copy(), conn[neg, 2].copy()
    fixed = np.nonzero(ijk[:, 0] == 0)[0].astype(np.int32)
    return TetBeam(nx, ny, nz, X, conn.astype(np.int32), fixed)


def hex_beam(a: int, b: int, c: int, spacing: float = SPACING, jitter: float = 0.0,
             seed: int = 1) -> HexBeam:
    """Beam of a x b x c trilinear hexes; optional seeded jitter U(-j, j)*spacing."""
    ny, nz, nx = a, b, c
    ijk, X = _grid_nodes(nx, ny, nz, spacing)
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        X = X + rng.uniform(-jitter, jitter, size=X.shape) * spacing
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cubes = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
    corder = np.argsort(cubes[:, 0] + nx * (cubes[:, 1] + ny * cubes[:, 2]))
    cubes = cubes[corder]
    cols = []
    for a_loc in range(8):
        dx, dy, dz = a_loc & 1, (a_loc >> 1) & 1, (a_loc >> 2) & 1
        cols.append(_node_id(nx, ny, cubes[:, 0] + dx, cubes[:, 1] + dy, cubes[:, 2] + dz))
    conn = np.stack(cols, axis=1).astype(np.int32)
    fixed = np.nonzero(ijk[:, 0] == 0)[0].astype(np.int32)
    return HexBeam(nx, ny, nz, X, conn, fixed)


# ---------------------------------------------------------------- dead loads

def end_face_tris(mesh: TetBeam) -> np.ndarray:
    """Tet faces lying on the grid face i = nx, as [n_tri, 3] node ids."""
    on_end = np.zeros(mesh.n_nodes, dtype=bool)
    ids = np.arange(mesh.n_nodes)
    on_end[(ids % (mesh.nx + 1)) == mesh.nx] = True
    tris = []
    for drop in range(4):
        f = np.delete(mesh.conn, drop, axis=1)
        sel = on_end[f].all(axis=1)
        tris.append(f[sel])
    return np.concatenate(tris, axis=0)


def end_face_quads(mesh: HexBeam) -> np.ndarray:
    """Hex faces on the grid face i = nx as [n_quad, 4] node ids in the
    bilinear order (dy, dz) = (0,0), (1,0), (0,1), (1,1)."""
    last = mesh.conn.reshape(mesh.nz, mesh.ny, mesh.nx, 8)[:, :, -1, :]
    quad = last[..., [1, 3, 5, 7]]  # dx = 1 corners, ordered by dy + 2 dz
    return quad.reshape(-1, 4)


def end_traction(mesh: TetBeam, traction: np.ndarray) -> np.ndarray:
    """Nodal shares [n_nodes, 3] of a uniform dead traction (force per rest
    area) on the end face x = L: a triangle gives area/3 to each vertex; a
    bilinear quad gives int N_a dA by 2x2 Gauss on its rest geometry."""
    t = np.asarray(traction, dtype=np.float64).reshape(3)
    out = np.zeros((mesh.n_nodes, 3))
    if mesh.elem_type == TET4:
        tri = end_face_tris(mesh)
        P = mesh.X[tri]
        area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
        share = np.repeat(area / 3.0, 3)
        np.add.at(out, tri.ravel(), share[:, None] * t[None, :])
    else:
        quad = end_face_quads(mesh)
        P = mesh.X[quad]                       # [nq, 4, 3]
        g = 1.0 / math.sqrt(3.0)
        for s in (-g, g):
            for r in (-g, g):
                N = 0.25 * np.array([(1 - s) * (1 - r), (1 + s) * (1 - r),
                                     (1 - s) * (1 + r), (1 + s) * (1 + r)])
                dNs = 0.25 * np.array([-(1 - r), (1 - r), -(1 + r), (1 + r)])
                dNr = 0.25 * np.array([-(1 - s), -(1 + s), (1 - s), (1 + s)])
                xs = np.einsum("a,qai->qi", dNs, P)
                xr = np.einsum("a,qai->qi", dNr, P)
                dA = np.linalg.norm(np.cross(xs, xr), axis=1)
                np.add.at(out, quad.ravel(), (dA[:, None] * N[None, :]).reshape(-1)[:, None] * t[None, :])
    return out


def body_force(mesh: TetBeam, rho: float, g) -> np.ndarray:
    """Nodal shares [n_nodes, 3] of a uniform dead body force rho*g:
    int rho N_a dV, i.e. rho*V/4 per tet vertex; 2x2x2 Gauss for hexes."""
    g = np.asarray(g, dtype=np.float64).reshape(3)
    out = np.zeros(mesh.n_nodes)
    if mesh.elem_type == TET4:
        d = mesh.X[mesh.conn[:, 1:]] - mesh.X[mesh.conn[:, [0]]]
        vol = np.einsum("ei,ei->e", d[:, 0], np.cross(d[:, 1], d[:, 2])) / 6.0
        np.add.at(out, mesh.conn.ravel(), np.repeat(rho * vol / 4.0, 4))
    else:
        P = mesh.X[mesh.conn]                  # [E, 8, 3]
        gp = 1.0 / math.sqrt(3.0)
        corner = np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1]
                           for a in range(8)], dtype=np.float64)
        for q in range(8):
            xi = corner[q] * gp
            N = np.prod(1.0 + corner * xi[None, :], axis=1) / 8.0
            dN = np.empty((8, 3))
            for r in range(3):
                o = [c for c in range(3) if c != r]
                dN[:, r] = corner[:, r] * (1 + corner[:, o[0]] * xi[o[0]]) * (1 + corner[:, o[1]] * xi[o[1]]) / 8.0
            J = np.einsum("eai,ar->eir", P, dN)
            detJ = np.linalg.det(J)
            np.add.at(out, mesh.conn.ravel(), (rho * detJ[:, None] * N[None, :]).ravel())
    return out[:, None] * g[None, :]


# ------------------------------------------------------------- the workloads

def lognormal_modulus(n: int, seed: int, median: float = 1e4, sigma: float = 0.3) -> np.ndarray:
    """Per-element Young's modulus median*exp(sigma*z), z ~ N(0,1) (PCG64 seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return median * np.exp(sigma * rng.standard_normal(n))


def batched_beams(n_beams: int = 64, seed: int = 7):
    """Uneven tet beams of the batched workload: cross-section m x m with
    m in [4, 12], target DOF D ~ U[2000, 40000], length from D, material SVK
    or neo-Hookean (p = 1/2), E ~ U[5e3, 5e4], nu ~ U[0.3, 0.49]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_beams):
        m = int(rng.integers(4, 13))
        D = float(rng.uniform(2000.0, 40000.0))
        L = max(1, int(round(D / (3.0 * (m + 1) ** 2))) - 1)
        while 3 * (m + 1) ** 2 * (L + 1) < 2000:
            L += 1
        while L > 1 and 3 * (m + 1) ** 2 * (L + 1) > 40000:
            L -= 1
        model = SVK if rng.uniform() < 0.5 else NEOHOOKE
        E = float(rng.uniform(5e3, 5e4))
        nu = float(rng.uniform(0.3, 0.49))
        out.append(dict(m=m, L=L, model=model, E=E, nu=nu))
    return out


@dataclasses.dataclass
class Workload:
    name: str
    mesh: TetBeam
    model: int
    params: np.ndarray      # [3] or [n_elems, 3]: (mu, lambda, 0) or (C10, C01, kappa)
    rho: float
    h: float
    alpha: float
    beta: float
    steps: int
    tol: float
    precision: int          # 0 FP64, 1 mixed
    refactor_every: int
    loads: callable         # step index -> p_t [n_nodes, 3]

    def p(self, step: int) -> np.ndarray:
        return self.loads(step)


def _tet0():
    mesh = tet_beam(4, 4, 16)
    mu, lam = lame_from_young(1e4, 0.45)
    grav = body_force(mesh, RHO, (0.0, 0.0, G_Z))
    return Workload("tet4x4x16-svk-fp64", mesh, SVK, np.array([mu, lam, 0.0]), RHO, H, ALPHA,
                    BETA, 10, 1e-10, 0, 1, lambda s: grav)


def _hex1(a=20, b=20, c=80):
    mesh = hex_beam(a, b, c, jitter=0.1, seed=1)
    trac = end_traction(mesh, (50.0, 0.0, 0.0))
    return Workload(f"hex{a}x{b}x{c}-nh", mesh, NEOHOOKE, np.array([3.4e3, 3.1e4, 0.0]), RHO, H,
                    ALPHA, BETA, 50, 1e-8, 1, 5, lambda s: trac)


def _tet2(a=30, b=30, c=120):
    mesh = tet_beam(a, b, c)
    grav = body_force(mesh, RHO, (0.0, 0.0, G_Z))
    unit = end_traction(mesh, (0.0, 0.0, 1.0))

    def loads(s):
        return grav + (100.0 * math.sin(2.0 * math.pi * (s * H) / 0.5)) * unit

    return Workload(f"tet{a}x{b}x{c}-mr", mesh, MOONEY_RIVLIN, np.array([1.5e3, 5e2, 5e4]), RHO, H,
                    ALPHA, BETA, 100, 1e-8, 1, 5, loads)


WORKLOADS = {
    "tet4x4x16-svk-fp64": _tet0,
    "hex20x20x80-nh": _hex1,
    "tet30x30x120-mr": _tet2,
}


def workload(name: str, **kw) -> Workload:
    """Named workload; size variants of the same family either by keyword
    (workload('tet-mr', a=4, b=4, c=16)) or by name ('tet20x20x80-mr',
    'hex8x8x32-nh')."""
    if name in WORKLOADS:
        return WORKLOADS[name]()
    import re
    m = re.fullmatch(r"(tet|hex)(\d+)x(\d+)x(\d+)-(mr|nh)", name)
    if m and (m.group(1), m.group(5)) in (("tet", "mr"), ("hex", "nh")):
        a, b, c = int(m.group(2)), int(m.group(3)), int(m.group(4))
        return _tet2(a, b, c) if m.group(1) == "tet" else _hex1(a, b, c)
    if name == "tet-mr":
        return _tet2(**kw)
    if name == "hex-nh":
        return _hex1(**kw)
    raise KeyError(name)


@dataclasses.dataclass
class BatchMember:
    mesh: TetBeam
    model: int
    params: np.ndarray      # [3]
    load: np.ndarray        # [n_nodes, 3] gravity dead load (constant in time)


def batch_workload(n_beams: int = 64, seed: int = 7):
    """Members of the batched workload (sizes and materials of batched_beams):
    tet beams m x m x L, SVK or neo-Hookean with (E, nu), clamped at x = 0,
    under a tenth of gravity (the most slender, softest members fold through
    themselves under full gravity within 25 steps), h / alpha / beta / rho of
    the other workloads."""
    out = []
    for spec in batched_beams(n_beams, seed):
        mesh = tet_beam(spec["m"], spec["m"], spec["L"])
        mu, lam = lame_from_young(spec["E"], spec["nu"])
        out.append(BatchMember(mesh, spec["model"], np.array([float(mu), float(lam), 0.0]),
                               body_force(mesh, RHO, (0.0, 0.0, 0.1 * G_Z))))
    return out
