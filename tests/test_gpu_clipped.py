"""Parity of the CUDA path with the FP64 oracle where a bounded lattice edge
cuts a marker's support (Eq. 14 with nodes outside the lattice dropped).

Bodies touch a free-slip wall row, a no-slip wall row (strips of markers
along the wall, and a cylinder resting on it), and the inlet and outlet
columns of a zero-gradient channel, so their 3- and 4-point supports lose a
row or a column: the interpolation weights of those markers no longer
sum to one (Eqs. 12, 14), the spread drops the same terms (Eqs. 13, 15), and
the boundary rules act on nodes that also carry IB force.  Each case runs
1000 steps on the oracle and, through the C ABI, on several collide-stream
kernel variants in both population layouts; the bars are those of the
cylinder cases (velocity relative L2 <= 1e-5 after the run, Cd and Cl
<= 1e-4 at every step, per-marker U* within 1e-5 U and F_b within 2e-5 U,
the force density of the last step within 1e-4 of its largest value), and
the variants must agree bitwise with each other.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1806_09403_gb300 import _build  # noqa: E402
from paper_1806_09403_gb300 import btdf as B  # noqa: E402

STEPS = 1000
VEL_TOL = 1e-5
CD_TOL = 1e-4
# (variant, layout): 4 and 2 nodes per lane, the TMA-tiled kernel, the
# prefetching 4-node kernel and the two warp-specialized TMA kernels, across
# both layouts
RUNS = [(1, B.LAYOUT_ROWS), (2, B.LAYOUT_PLANES), (3, B.LAYOUT_ROWS), (11, B.LAYOUT_PLANES),
        (9, B.LAYOUT_ROWS), (12, B.LAYOUT_PLANES), (13, B.LAYOUT_ROWS)]


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    O.set_threads(min(os.cpu_count() or 1, 32))


def strips_case(bc_y, delta):
    """160 x 64 channel, tau = 0.56.  A strip of 40 markers (ds = dh) 0.3
    above row 0 and another 0.35 below row ny-1, so the support of every
    marker reaches one row beyond the wall.  On free-slip walls the strips
    are at rest (no-slip patches on a slip wall); on no-slip walls they move
    along the wall (U_b = 0.5 U below, -0.3 U above, belts)."""
    c = W.Case(f"strips{bc_y}_d{delta}", 160, 64, 0.56, W.U_IN, delta, W.BCX_INOUT, bc_y,
               seed=21 + bc_y, D=16.0)
    ub = (0.0, 0.0) if bc_y == W.BCY_FREESLIP else (0.5 * W.U_IN, -0.3 * W.U_IN)
    for x0, y, u in ((40.25, 0.3, ub[0]), (100.4, 63.0 - 0.35, ub[1])):
        c.bodies.append(W.Body(X=np.arange(40) + x0, Y=np.full(40, y), ds=1.0,
                               Ubx=np.full(40, u), Uby=np.zeros(40), D=16.0))
    return c


def wall_cylinder_case(bc_y, delta):
    """160 x 80 channel, tau = 0.56; a cylinder (D = 16, 50 markers) whose
    lowest marker sits 0.3 above row 0."""
    c = W.Case(f"wallcyl{bc_y}_d{delta}", 160, 80, 0.56, W.U_IN, delta, W.BCX_INOUT, bc_y,
               seed=21 + bc_y, D=16.0)
    c.bodies.append(W.circle_markers(48.37, 8.3, 16.0, 50))
    return c


def columns_case(delta):
    """160 x 64 zero-gradient channel.  A line of 45 markers (ds = dh) at
    x = 0.3, just right of the inlet column, prescribes a shaped inflow
    U_b = U (1 + 0.3 sin(2 pi (y - 10) / 45)), 0) (a cylinder at rest there
    fights the inlet rule and drives the density below 0.5); a cylinder's
    rightmost marker sits 0.3 right of the outlet column x = nx-1."""
    c = W.Case(f"columns_d{delta}", 160, 64, 0.6, W.U_IN, delta, W.BCX_INOUT, W.BCY_FREESLIP,
               seed=31, D=16.0)
    Y = np.arange(10.0, 55.0) + 0.21
    ub = W.U_IN * (1.0 + 0.3 * np.sin(2.0 * np.pi * (Y - 10.0) / 45.0))
    c.bodies.append(W.Body(X=np.full(len(Y), 0.3), Y=Y, ds=1.0, Ubx=ub, Uby=np.zeros(len(Y)),
                           D=16.0))
    c.bodies.append(W.circle_markers(159.3 - 8.0, 36.41, 16.0, 50))
    return c


CASES = {
    "freeslip_strips": lambda d: strips_case(W.BCY_FREESLIP, d),
    "noslip_belts": lambda d: strips_case(W.BCY_NOSLIP, d),
    "freeslip_cylinder": lambda d: wall_cylinder_case(W.BCY_FREESLIP, d),
    "noslip_cylinder": lambda d: wall_cylinder_case(W.BCY_NOSLIP, d),
    "inlet_outlet_columns": columns_case,
}


def clipped_markers(case, body):
    """Markers of a body whose support leaves the lattice (counted on the
    host from the support rule |x_e - X| < w/2 alone)."""
    w = {2: 2, 3: 3, 4: 4, 5: 4}[case.delta]
    b = case.bodies[body]
    lo_x = np.floor(b.X - 0.5 * w) + 1
    lo_y = np.floor(b.Y - 0.5 * w) + 1
    out_x = (lo_x < 0) | (lo_x + w - 1 > case.nx - 1)
    out_y = (lo_y < 0) | (lo_y + w - 1 > case.ny - 1)
    return int(np.count_nonzero(out_x | out_y))


@pytest.fixture(scope="module")
def oracle_runs():
    cache = {}

    def get(name, delta):
        key = (name, delta)
        if key not in cache:
            case = CASES[name](delta)
            sim = O.Sim.from_case(case)
            sim.step(STEPS)
            R, UX, UY = sim.moments()
            hist = [sim.history(b, 0, STEPS) for b in range(len(case.bodies))]
            diag = [sim.marker_diag(b) for b in range(len(case.bodies))]
            cache[key] = (case, (R, UX, UY), hist, diag, sim.force_field())
        return cache[key]

    return get


@pytest.mark.parametrize("delta", [3, 4])
@pytest.mark.parametrize("name", list(CASES))
def test_clipped_support_against_oracle(name, delta, oracle_runs):
    case, (R, UX, UY), hist, diag, (FX, FY) = oracle_runs(name, delta)
    assert all(clipped_markers(case, b) > 0 for b in range(len(case.bodies)))
    q = 0.5 * case.u_in ** 2 * case.D
    outs = []
    for variant, layout in RUNS:
        lat = B.Lattice.from_case(case, layout=layout, history_len=STEPS)
        lat.tune(variant, 0)
        lat.step(STEPS)
        lat.sync()
        r, ux, uy = lat.moments()
        num = ((ux - UX) ** 2 + (uy - UY) ** 2).sum()
        e = float(np.sqrt(num / (UX ** 2 + UY ** 2).sum()))
        assert e <= VEL_TOL, f"variant {variant}: velocity rel L2 {e:.3e}"
        assert float(np.abs(r - R).max()) <= 1e-5
        for b in range(len(case.bodies)):
            gx, gy = lat.forces(b, 0, STEPS)
            rx, ry = hist[b]
            CD, CL = rx / q, ry / q
            scale = np.abs(CD).mean()
            ecd = np.abs(gx / q - CD) / np.maximum(np.abs(CD), scale)
            ecl = np.abs(gy / q - CL) / np.maximum(np.maximum(np.abs(CL), np.abs(CD)), scale)
            assert ecd.max() <= CD_TOL, f"variant {variant} body {b}: Cd err {ecd.max():.3e}"
            assert ecl.max() <= CD_TOL, f"variant {variant} body {b}: Cl err {ecl.max():.3e}"
            m = lat.markers(b)
            d = diag[b]
            assert np.abs(m["Usx"] - d["Usx"]).max() <= 1e-5 * case.u_in
            assert np.abs(m["Usy"] - d["Usy"]).max() <= 1e-5 * case.u_in
            assert np.abs(m["Fbx"] - d["Fbx"]).max() <= 2e-5 * case.u_in
            assert np.abs(m["Fby"] - d["Fby"]).max() <= 2e-5 * case.u_in
        gfx, gfy = lat.field(B.FIELD_FX), lat.field(B.FIELD_FY)
        s = max(np.abs(FX).max(), np.abs(FY).max())
        assert np.abs(gfx - FX).max() <= 1e-4 * s and np.abs(gfy - FY).max() <= 1e-4 * s
        outs.append((lat.field(B.FIELD_POPS), lat.forces(0)[0]))
        lat.close()
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


def test_clipped_support_drops_the_outside_weight():
    """The spread of a clipped body puts no force outside the lattice and
    keeps only the inside share of Eq. 27: the force density summed over the
    lattice is below sum_l F_l ds drs in magnitude by the clipped weights,
    on both sides alike."""
    case = strips_case(W.BCY_FREESLIP, 4)
    case.bodies = case.bodies[:1]
    lat = B.Lattice.from_case(case, history_len=64)
    sim = O.Sim.from_case(case)
    lat.step(40)
    sim.step(40)
    gfx = lat.field(B.FIELD_FX).astype(np.float64)
    FX, _ = sim.force_field()
    Fp, _ = sim.history(0, 39, 1)
    assert abs(gfx.sum() - FX.sum()) <= 1e-5 * np.abs(FX).sum()
    # the row below the wall held delta(-1.3) of every marker's y weight: the
    # force density keeps sum_l F_l ds drs (1 - delta(-1.3)), not all of it
    d = O.delta(4, -1.3)
    assert abs(FX.sum() + Fp[0] * (1.0 - d)) <= 1e-6 * abs(Fp[0])
    assert abs(FX.sum() + Fp[0]) > 0.5 * d * abs(Fp[0])
