"""Parity at the full sizes of the benchmarked configurations, in the launch
configurations bench.py times (CUDA-graph replay; on the 8192 x 4096 lattice
the collide-stream variant its autotuner keeps and the library's automatic
choice, 11 for FP32 and the warp-specialized TMA kernel 12 for FP16 / BF16,
each also checked bitwise against a register kernel with one row segment per
warp, 2 for FP32 and 1 for FP16 / BF16):

* the 8192 x 4096 lattice with 400 cylinders (D = 20, 63 markers each),
  FP32, against the FP64 oracle over 100 steps: velocity field and the drag
  and lift of every one of the 400 bodies (velocity 1e-5, Cd and Cl 1e-4);
  FP16 and BF16 storage on the same lattice against the same oracle run:
  the drag and lift series of every body within 1 % (relative L2 over the
  100 steps, lift on the drag scale: the bar of the mixed-precision form);
* the 512-lattice batch (lattices of 128 x 64 .. 1024 x 512): four sampled
  lattices against the oracle over 200 steps;
* the 800 x 400 adjoint window (500 steps after 2000, checkpoint every 50):
  dJ/dU against central differences of the FP64 oracle (eps = 1e-4), which
  starts from the oracle's own state after the same 2000 steps;
* the largest lattice the 32-bit element offsets allow, by translation
  invariance against a small lattice.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1806_09403_gb300 import _build  # noqa: E402
from paper_1806_09403_gb300 import btdf as B  # noqa: E402
from paper_1806_09403_gb300.autograd import DragWindow  # noqa: E402

VEL_TOL = 1e-5
CD_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    O.set_threads(min(os.cpu_count() or 1, 64))


def vel_err(lat, sim):
    _, ux, uy = lat.moments()
    _, rx, ry = sim.moments()
    num = ((ux.astype(np.float64) - rx) ** 2 + (uy.astype(np.float64) - ry) ** 2).sum()
    return float(np.sqrt(num / (rx ** 2 + ry ** 2).sum()))


def force_err(gx, gy, rx, ry):
    """Largest per-step Cd / Cl error on the drag scale (the bars of the
    cylinder parity tests)."""
    scale = np.abs(rx).mean()
    ecd = np.abs(gx - rx) / np.maximum(np.abs(rx), scale)
    ecl = np.abs(gy - ry) / np.maximum(np.maximum(np.abs(ry), np.abs(rx)), scale)
    return float(ecd.max()), float(ecl.max())


@pytest.fixture(scope="module")
def many_cylinders_oracle():
    case = W.many_cylinders()
    sim = O.Sim.from_case(case)
    sim.step(100)
    hist = [sim.history(b, 0, 100) for b in range(len(case.bodies))]
    return case, sim, hist


def worst_force_err(lat, case, hist):
    fx, fy = lat.forces(-1, 0, 100)     # every body, step-major
    worst = (0.0, 0.0)
    for b in range(len(case.bodies)):
        rx, ry = hist[b]
        ecd, ecl = force_err(fx[:, b], fy[:, b], rx, ry)
        worst = (max(worst[0], ecd), max(worst[1], ecl))
    return worst


def run_variant(case, storage, variant):
    lat = B.Lattice.from_case(case, storage=storage, history_len=128)
    if variant:
        lat.tune(variant, 0)
    lat.step(100)
    return lat


def same_bits(a, b):
    """Velocity fields and every body's force series of two runs agree bit for bit."""
    for kind in (B.FIELD_UX, B.FIELD_UY):
        assert np.array_equal(a.field(kind), b.field(kind))
    fa, fb = a.forces(-1, 0, 100), b.forces(-1, 0, 100)
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])


def test_many_cylinders_8192x4096_100_steps(many_cylinders_oracle):
    case, sim, hist = many_cylinders_oracle
    lat = run_variant(case, B.BTDF_F32, 11)
    same_bits(lat, run_variant(case, B.BTDF_F32, 2))
    e = vel_err(lat, sim)
    worst = worst_force_err(lat, case, hist)
    print(f"\n[8192x4096, 400 cylinders, 100 steps] velocity rel L2 {e:.2e}, "
          f"worst Cd {worst[0]:.2e}, worst Cl {worst[1]:.2e} over 400 bodies")
    assert e <= VEL_TOL
    assert worst[0] <= CD_TOL and worst[1] <= CD_TOL


@pytest.mark.parametrize("storage,name", [(B.BTDF_F16DEV, "f16"), (B.BTDF_BF16DEV, "bf16")])
def test_many_cylinders_8192x4096_mixed_precision(many_cylinders_oracle, storage, name):
    case, sim, hist = many_cylinders_oracle
    lat = run_variant(case, storage, 12)
    same_bits(lat, run_variant(case, storage, 1))
    e = vel_err(lat, sim)
    fx, fy = lat.forces(-1, 0, 100)
    ecd = ecl = 0.0
    for b in range(len(case.bodies)):
        rx, ry = hist[b]
        ecd = max(ecd, float(np.linalg.norm(fx[:, b] - rx) / np.linalg.norm(rx)))
        ecl = max(ecl, float(np.linalg.norm(fy[:, b] - ry) / np.linalg.norm(rx)))
    worst = worst_force_err(lat, case, hist)
    print(f"\n[8192x4096, 400 cylinders, 100 steps, {name}] velocity rel L2 {e:.2e}, "
          f"worst body: Cd series {ecd:.2e}, Cl series {ecl:.2e} (rel L2); worst single step "
          f"Cd {worst[0]:.2e}, Cl {worst[1]:.2e}")
    assert ecd <= 1e-2 and ecl <= 1e-2


def test_batch_512_sampled_lattices():
    cases = W.batch_cases(512, seed=7)
    bt = B.Batch.from_cases(cases, history_len=256)
    bt.step(200)
    first_body = np.cumsum([0] + [len(c.bodies) for c in cases])
    sample = [0, 137, 301, 511]
    for i in sample:
        c = cases[i]
        sim = O.Sim.from_case(c)
        sim.step(200)
        _, rx, ry = sim.moments()
        ux, uy = bt.field(i, B.FIELD_UX), bt.field(i, B.FIELD_UY)
        e = float(np.sqrt((((ux - rx) ** 2 + (uy - ry) ** 2).sum()) / ((rx ** 2 + ry ** 2).sum())))
        gx, gy = bt.forces(int(first_body[i]), 0, 200)
        hx, hy = sim.history(0, 0, 200)
        ecd, ecl = force_err(gx, gy, hx, hy)
        print(f"\n[batch lattice {i}: {c.nx}x{c.ny}, Re {c.Re:g}] velocity {e:.2e}, Cd {ecd:.2e}, Cl {ecl:.2e}")
        assert e <= max(VEL_TOL, 200 * 2.0 ** -24)
        assert ecd <= CD_TOL and ecl <= CD_TOL


def test_adjoint_800x400_inflow_gradient_against_fp64():
    case = W.adjoint_cylinder()
    t0, n, eps = 2000, 500, 1e-4
    lat = B.Lattice.from_case(case, history_len=256)
    lat.step(t0)
    win = DragWindow.for_lattice(lat, 200.0, 200.0, 0.5 * case.D, n, every=50, dref=case.D)
    z = np.zeros(len(case.bodies[0].X))
    J = win.evaluate(case.u_in, z)
    dU, _ = win.gradients(case.u_in, z)

    base = O.Sim.from_case(case)
    base.step(t0)
    start = base.pops()
    b = case.bodies[0]

    def window(u):
        s = O.Sim(case.nx, case.ny, case.tau, u, case.bc_x, case.bc_y, 0.0, 0.0, case.delta, case.nf)
        s.init_fields(*case.initial_fields())
        s.set_pops(start)
        s.apply_inlet()
        s.add_body(b.X, b.Y, b.ds, drs=case.drs)
        s.step(n)
        fx, _ = s.history(0)
        return float(np.mean(fx) / (0.5 * u * u * case.D))

    J64 = window(case.u_in)
    fd = (window(case.u_in + eps) - window(case.u_in - eps)) / (2 * eps)
    print(f"\n[800x400 adjoint] J {J:.8f} (FP64 {J64:.8f}); dJ/dU adjoint {dU:.6e}, FP64 FD {fd:.6e} "
          f"({abs(dU / fd - 1):.1e})")
    assert abs(J / J64 - 1) <= 1e-4
    assert abs(dU / fd - 1) <= 1e-3


def test_largest_lattice_32bit_offsets():
    """The largest lattice of width 32768 the 32-bit element offsets allow
    (32768 x 14563: 9 x nxp x ny just below 2^32, 34 GB of FP32 populations),
    fully periodic, uniform flow, one cylinder near the far corner where the
    offsets are largest.  Translation invariance: after 20 steps the flow
    around that cylinder equals the flow around the same cylinder (same
    fractional position) in a 128 x 128 periodic lattice, and the lattice far
    from it is still the uniform state."""
    nx, ny, tau, u = 32768, 14563, 0.6, (0.03, 0.01)
    d, n = 16.0, 50
    cx, cy = nx - 60.3, ny - 60.7
    big = B.Lattice(nx, ny, tau, 0.0, 3, 1, B.BTDF_F32, B.BTDF_BCX_PERIODIC, B.BTDF_BCY_PERIODIC,
                    history_len=32)
    big.init_fields(np.ones((ny, nx)), np.full((ny, nx), u[0]), np.full((ny, nx), u[1]))
    big.add_cylinder(cx, cy, d, n)
    ox, oy = nx - 128, ny - 128            # the small lattice is this window
    small = B.Lattice(128, 128, tau, 0.0, 3, 1, B.BTDF_F32, B.BTDF_BCX_PERIODIC, B.BTDF_BCY_PERIODIC,
                      history_len=32)
    small.init_fields(np.ones((128, 128)), np.full((128, 128), u[0]), np.full((128, 128), u[1]))
    small.add_cylinder(cx - ox, cy - oy, d, n)
    big.step(20)
    small.step(20)
    dev = torch.empty((ny, nx), dtype=torch.float32, device="cuda")
    for kind in (B.FIELD_UX, B.FIELD_UY, B.FIELD_RHO):
        big.field_to_device(kind, dev.data_ptr())
        torch.cuda.synchronize()
        win = dev[oy:, ox:].cpu().numpy()
        ref = small.field(kind)
        # the cylinder and the 20-node front around it lie inside the window
        inner = (slice(16, 128), slice(16, 128))
        np.testing.assert_allclose(win[inner], ref[inner], rtol=0, atol=2e-7)
        far = dev[: ny // 2, : nx // 2]
        val = {B.FIELD_UX: u[0], B.FIELD_UY: u[1], B.FIELD_RHO: 1.0}[kind]
        assert float((far - val).abs().max()) < 1e-6
    del dev
    fb, fs = big.forces(0), small.forces(0)
    np.testing.assert_allclose(fb[0], fs[0], rtol=1e-5)
    big.close()

