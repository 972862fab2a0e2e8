"""Workload definitions: mesh, material, boundary conditions, loads, load path.

Only inputs live here.  The four workloads are the structured-box problems
the performance study runs (plane-strain P1 and P2 triangles, Q1 hexahedra,
P2 tetrahedra), each at a caller-chosen mesh size so that tests can run them
small and the benchmark at full size.

External loads are uniform tractions; their consistent nodal values come from
the closed-form per-face distributions of a constant load over a face element
(2-node edge 1/2,1/2; 3-node edge 1/6,2/3,1/6; 4-node square 1/4 each; 3-node
triangle 1/3 each; 6-node triangle 0 at vertices, 1/3 at midsides; 8-node
serendipity square -1/12 at corners, 1/3 at midsides), times the face measure.
The oracle integrates the same loads by quadrature and a test checks that the
two agree.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .meshes import Mesh, boundary_nodes, structured_mesh, top_faces

# models, as in the C-ABI enumeration
ELASTIC, VM_KIN, VM_ISO, DP = 0, 1, 2, 3

_FACE_WEIGHTS = {
    "L1": np.array([1 / 2, 1 / 2]),
    "L2": np.array([1 / 6, 1 / 6, 2 / 3]),            # (end, end, mid)
    "S1": np.array([1 / 4] * 4),
    "S2": np.array([-1 / 12] * 4 + [1 / 3] * 4),
    "T1": np.array([1 / 3] * 3),
    "T2": np.array([0.0] * 3 + [1 / 3] * 3),
}


@dataclass
class Material:
    model: int
    E: float
    nu: float
    Y: float = 0.0        # von Mises yield value (Frobenius norm of the deviator)
    H: float = 0.0        # von Mises hardening modulus (kinematic a or isotropic H)
    c0: float = 0.0       # Drucker-Prager cohesion
    phi: float = 0.0      # friction angle [rad]
    psi: float = 0.0      # dilatancy angle [rad]
    Hc: float = 0.0       # linear cohesion-hardening modulus


@dataclass
class Problem:
    name: str
    mesh: Mesh
    material: Material
    dirichlet: np.ndarray      # uint8 [n_n*dim], 1 = prescribed
    u_D_unit: np.ndarray       # float64 [n_n*dim], prescribed values at zeta = 1
    f_unit: np.ndarray         # float64 [n_n*dim], external load at zeta = 1
    zeta: np.ndarray           # float64 [n_steps], load factors of the path
    newton_rtol: float = 1e-10
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return self.mesh.dim

    @property
    def n_dof(self) -> int:
        return self.mesh.n_nodes * self.mesh.dim


def traction_load(mesh: Mesh, traction) -> np.ndarray:
    """Consistent nodal load [n_n*dim] of a uniform traction vector on the top face."""
    kind, faces = top_faces(mesh)
    w = _FACE_WEIGHTS[kind]
    x = mesh.coords[faces]                     # [n_f][n_fn][dim]
    if mesh.dim == 2:
        meas = np.abs(x[:, 1, 0] - x[:, 0, 0])  # straight horizontal edges
    else:
        c = x[:, :3 if kind.startswith("T") else 4, :2]
        if kind.startswith("T"):
            a, b = c[:, 1] - c[:, 0], c[:, 2] - c[:, 0]
            meas = 0.5 * np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
        else:
            meas = np.abs((c[:, 1, 0] - c[:, 0, 0]) * (c[:, 3, 1] - c[:, 0, 1]))
    f = np.zeros((mesh.n_nodes, mesh.dim))
    contrib = meas[:, None] * w[None, :]
    for a in range(mesh.dim):
        np.add.at(f[:, a], faces.ravel(), (contrib * traction[a]).ravel())
    return f.ravel()


def _mask(mesh: Mesh, pairs) -> np.ndarray:
    """Dirichlet mask from (axis_of_face, side, component) triples."""
    m = np.zeros((mesh.n_nodes, mesh.dim), dtype=np.uint8)
    for axis, side, comp in pairs:
        m[boundary_nodes(mesh, axis, side), comp] = 1
    return m.ravel()


def first_yield_traction_vm(E, nu, Y):
    """Traction at first yield of the homogeneous plane-strain column (sigma_xx=0)."""
    sig_eq = Y * math.sqrt(1.5)
    return sig_eq / math.sqrt(1.0 - nu + nu * nu)


def plane_strain_limit_traction_dp(c0, phi):
    """Limit traction 2c/(1-eta) of the homogeneous plane-strain column, psi = 0."""
    t = math.tan(phi)
    q = math.sqrt(9.0 + 12.0 * t * t)
    eta, c = 3.0 * t / q, 3.0 * c0 / q
    return 2.0 * c / (1.0 - eta)


def plane_column(elem_type: str, n: int, material: Material, t_max: float, n_steps: int) -> Problem:
    """[0,10]^2, u_x = 0 on x = 0, u_y = 0 on y = 0, compressive traction on y = 10."""
    mesh = structured_mesh(elem_type, 2, (n, n), (10.0, 10.0))
    dirichlet = _mask(mesh, [(0, "min", 0), (1, "min", 1)])
    f_unit = traction_load(mesh, (0.0, -t_max))
    zeta = np.arange(1, n_steps + 1, dtype=np.float64) / n_steps
    return Problem(f"plane_column_{elem_type}_{n}", mesh, material, dirichlet,
                   np.zeros(mesh.n_nodes * 2), f_unit, zeta)


def vm_iso_material():
    return Material(VM_ISO, E=206900.0, nu=0.29, Y=450.0 * math.sqrt(2.0 / 3.0), H=10000.0)


def p1_plane_vm(n: int = 20, n_steps: int = 20) -> Problem:
    """P1 triangles, von Mises with isotropic hardening, to 1.5x first yield."""
    mat = vm_iso_material()
    t_y = first_yield_traction_vm(mat.E, mat.nu, mat.Y)
    p = plane_column("P1", n, mat, 1.5 * t_y, n_steps)
    p.newton_rtol = 1e-12
    p.extra["t_first_yield"] = t_y
    return p


def p2_plane_dp(n: int = 256, n_steps: int = 40, load_fraction: float = 0.98) -> Problem:
    """P2 triangles (7-point rule), nonassociated Drucker-Prager (psi = 0), to load_fraction * t_lim.

    With psi = 0 the plane-strain tangent of the homogeneous column becomes
    singular at t_lim (the uniform plastic flow mode satisfies the supports);
    at 0.98 t_lim the last step's tangent has eigenvalues with negative real
    parts, which the solver meets with a sparse LU.
    """
    mat = Material(DP, E=206900.0, nu=0.29, c0=450.0, phi=math.radians(20.0), psi=0.0, Hc=0.0)
    t_lim = plane_strain_limit_traction_dp(mat.c0, mat.phi)
    p = plane_column("P2", n, mat, load_fraction * t_lim, n_steps)
    p.extra["t_lim"] = t_lim
    p.extra["load_fraction"] = load_fraction
    return p


def q1_cube_vm(n: int = 64, n_steps: int = 30, p_max: float = 675.0) -> Problem:
    """Q1 hexahedra on [0,10]^3, fixed base, pressure on the top face."""
    mesh = structured_mesh("Q1", 3, (n, n, n), (10.0, 10.0, 10.0))
    dirichlet = _mask(mesh, [(2, "min", 0), (2, "min", 1), (2, "min", 2)])
    f_unit = traction_load(mesh, (0.0, 0.0, -p_max))
    zeta = np.arange(1, n_steps + 1, dtype=np.float64) / n_steps
    return Problem(f"q1_cube_vm_{n}", mesh, vm_iso_material(), dirichlet,
                   np.zeros(mesh.n_nodes * 3), f_unit, zeta)


def p2_tet_strip_dp(n: int = 48, n_steps: int = 50, u_max: float = 0.1,
                    strip: float = 1.0) -> Problem:
    """P2 tetrahedra (6 per cube), DP with cohesion hardening, rigid strip on top."""
    mesh = structured_mesh("P2", 3, (n, n, n), (10.0, 10.0, 10.0))
    pairs = [(0, "min", 0), (0, "max", 0), (1, "min", 1), (1, "max", 1), (2, "min", 2)]
    dirichlet = _mask(mesh, pairs).reshape(-1, 3)
    u_D = np.zeros((mesh.n_nodes, 3))
    top = boundary_nodes(mesh, 2, "max")
    under = top[mesh.coords[top, 0] <= strip + 1e-9]
    dirichlet[under, 2] = 1
    u_D[under, 2] = -u_max
    mat = Material(DP, E=1e4, nu=0.3, c0=10.0, phi=math.radians(30.0), psi=math.radians(10.0),
                   Hc=1e3)
    zeta = np.arange(1, n_steps + 1, dtype=np.float64) / n_steps
    return Problem(f"p2_tet_strip_dp_{n}", mesh, mat, dirichlet.ravel(), u_D.ravel(),
                   np.zeros(mesh.n_nodes * 3), zeta)


def generic_box(elem_type: str, dim: int, n: int, material: Material, t_max: float,
                n_steps: int = 4) -> Problem:
    """Any element family on a box: column supports and a compressive top traction."""
    if dim == 2:
        return plane_column(elem_type, n, material, t_max, n_steps)
    mesh = structured_mesh(elem_type, 3, (n, n, n), (10.0, 10.0, 10.0))
    dirichlet = _mask(mesh, [(0, "min", 0), (1, "min", 1), (2, "min", 2)])
    f_unit = traction_load(mesh, (0.0, 0.0, -t_max))
    zeta = np.arange(1, n_steps + 1, dtype=np.float64) / n_steps
    return Problem(f"box_{elem_type}{dim}d_{n}", mesh, material, dirichlet,
                   np.zeros(mesh.n_nodes * 3), f_unit, zeta)


def batch_problems(seed: int = 1805, n_problems: int = 64, sizes=(16, 96), scale: float = 0.3,
                   families=None, n_steps: int = 10):
    """The batched sweep: independent problems with mesh sizes drawn uniformly from `sizes` elements
    per side and E, nu, Y, H each drawn from [1 - scale, 1 + scale] times the P1-column material;
    half 2D (P1 and P2 columns), half 3D (Q1 cubes).  Returns {family: [problems]} (one batch per
    element type), deterministic in `seed`."""
    g = np.random.default_rng(seed)
    fams = families or (["P1"] * (n_problems // 4) + ["P2"] * (n_problems // 4)
                        + ["Q1"] * (n_problems - 2 * (n_problems // 4)))
    base = vm_iso_material()
    out: dict = {}
    for i, fam in enumerate(fams):
        n = int(g.integers(sizes[0], sizes[1] + 1))
        f = g.uniform(1 - scale, 1 + scale, 4)
        nu = min(0.45, base.nu * f[1])
        mat = Material(VM_ISO, E=base.E * f[0], nu=nu, Y=base.Y * f[2], H=base.H * f[3])
        if fam == "Q1":
            p = q1_cube_vm(n=n, n_steps=n_steps)
            p.material = mat
        else:
            t_y = first_yield_traction_vm(mat.E, mat.nu, mat.Y)
            p = plane_column(fam, n, mat, 1.5 * t_y, n_steps)
        p.name = f"batch{i}_{fam}_{n}"
        out.setdefault(fam, []).append(p)
    return out


def l_shape_vm(elem_type: str = "Q2", m: int = 20, n_steps: int = 40, f_max: float = 200.0) -> Problem:
    """The L-shaped body of the von Mises experiment (Section 8.2): [0,10]^2 without the square
    [0,5)^2, m cells per side of each of its three squares; rollers on the left (x = 0) and bottom
    (y = 0) sides, a normal traction zeta(t) f_max on the top side, zeta rising linearly from 0 to 1
    on t in [0, 1], falling to -1 at t = 3 and returning to 0 at t = 4 (n_steps equal time steps);
    von Mises with linear kinematic hardening a = 1e4, Y = 450 sqrt(2/3), E = 206900, nu = 0.29."""
    box = structured_mesh(elem_type, 2, (2 * m, 2 * m), (10.0, 10.0))
    cent = box.coords[box.elem].mean(axis=1)
    keep = ~((cent[:, 0] < 5.0) & (cent[:, 1] < 5.0))
    elem = box.elem[keep]
    used = np.unique(elem)
    remap = -np.ones(box.n_nodes, dtype=np.int64)
    remap[used] = np.arange(len(used))
    mesh = Mesh(elem_type, 2, box.coords[used].copy(), remap[elem].astype(np.int32), box.shape, box.size)
    dirichlet = _mask(mesh, [(0, "min", 0), (1, "min", 1)])
    f_unit = traction_load(mesh, (0.0, f_max))
    t = np.arange(1, n_steps + 1, dtype=np.float64) * (4.0 / n_steps)
    zeta = np.where(t <= 1.0, t, np.where(t <= 3.0, 2.0 - t, t - 4.0))
    mat = Material(VM_KIN, E=206900.0, nu=0.29, Y=450.0 * math.sqrt(2.0 / 3.0), H=1e4)
    p = Problem(f"l_shape_vm_{elem_type}_{m}", mesh, mat, dirichlet, np.zeros(mesh.n_nodes * 2), f_unit, zeta)
    p.extra["f_max"] = f_max
    return p


def strip_footing_dp(elem_type: str = "P2", n: int = 160, footing: float = 1.0) -> Problem:
    """The strip-footing benchmark of the Drucker-Prager experiment (Section 8.3): [0,10]^2, rollers
    on the left, right and bottom sides, a footing of width `footing` at the top-left corner pushed
    down by the prescribed vertical displacement u_D = zeta (u_D_unit = -1 under the footing, zeta
    from 0 to 1); associated Drucker-Prager, perfectly plastic, E = 1e7, nu = 0.48, c0 = 450,
    phi = pi/9.  The default zeta is a uniform path; the paper doubles the increment adaptively
    (paper_1805_04155_gb300.drivers)."""
    mesh = structured_mesh(elem_type, 2, (n, n), (10.0, 10.0))
    dirichlet = _mask(mesh, [(0, "min", 0), (0, "max", 0), (1, "min", 1)]).reshape(-1, 2)
    u_D = np.zeros((mesh.n_nodes, 2))
    top = boundary_nodes(mesh, 1, "max")
    under = top[mesh.coords[top, 0] <= footing + 1e-9]
    dirichlet[under, 1] = 1
    u_D[under, 1] = -1.0
    mat = Material(DP, E=1e7, nu=0.48, c0=450.0, phi=math.pi / 9.0, psi=math.pi / 9.0)
    zeta = np.linspace(0.001, 0.01, 10)
    p = Problem(f"strip_footing_dp_{elem_type}_{n}", mesh, mat, dirichlet.ravel(), u_D.ravel(),
                np.zeros(mesh.n_nodes * 2), zeta)
    p.extra["footing"] = footing
    p.extra["footing_nodes"] = under
    return p


def prandtl_nc(phi: float) -> float:
    """Prandtl's bearing-capacity factor N_c = (N_q - 1) cot(phi), N_q = exp(pi tan phi) tan^2(pi/4 +
    phi/2): limit pressure c N_c of a smooth strip footing on a weightless Mohr-Coulomb half-space
    (the classical closed form the strip-footing benchmark approaches)."""
    nq = math.exp(math.pi * math.tan(phi)) * math.tan(math.pi / 4.0 + phi / 2.0) ** 2
    return (nq - 1.0) / math.tan(phi)


WORKLOADS = {
    "p1_plane_vm": p1_plane_vm,
    "p2_plane_dp": p2_plane_dp,
    "q1_cube_vm": q1_cube_vm,
    "p2_tet_strip_dp": p2_tet_strip_dp,
    "l_shape_vm": l_shape_vm,
    "strip_footing_dp": strip_footing_dp,
}
