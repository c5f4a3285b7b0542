"""Seeded synthetic workloads for the implicit FE step (mesh, materials, loads).

This module is shared by the CUDA path's tests/bench and by the FP64 oracle.
It holds *no* arithmetic of the method itself (no element force, tangent,
mass matrix, assembly or solve): only grid generation, connectivity,
orientation of the generated tets, seeded jitter and random draws, and the
nodal shares of dead external loads (body force and surface traction), which
the paper treats as the given external force vector p_t (Eq. "newton's law",
Section 3.2).

Conventions (all fixed here once, used by both sides):
  * a beam "a x b x c" has ny=a, nz=b, nx=c cubes; the long axis is x;
  * node (i, j, k) has index i + (nx+1) * (j + (ny+1) * k) and rest position
    (i, j, k) * spacing (+ optional seeded jitter);
  * DOF = 3 * node + component;
  * each cube (x-fastest order) is split into 6 Kuhn tets, one per axis
    permutation in lexicographic order (012, 021, 102, 120, 201, 210), the tet
    being (v0, v0+e_p0, v0+e_p0+e_p1, v0+1); its last two vertices are swapped
    when its signed volume is negative;
  * hex local node order a = dx + 2 dy + 4 dz;
  * the clamped set is the grid face i = 0 (selected by index, not coordinate).
"""
from .beams import (  # noqa: F401
    TetBeam, HexBeam, tet_beam, hex_beam, body_force, end_traction,
    end_face_tris, end_face_quads, lame_from_young, WORKLOADS, workload,
    batched_beams, batch_workload, BatchMember, lognormal_modulus, SVK, NEOHOOKE, MOONEY_RIVLIN, COROTATIONAL, TET4, HEX8,
)
