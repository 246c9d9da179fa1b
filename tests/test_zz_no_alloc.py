"""The IB force stage for callers that cannot allocate device memory.

Code that runs inside another framework's memory budget (a caching allocator
owns the device memory) and real-time loops that must not enter the driver's
allocator cannot call cudaMalloc.  They use btdf_ib_forces_static, whose
scratch is a fixed file-scope device array.  Here it must agree with the
regular path: a context's own IB stage applied to the same populations, for
every storage format, both population layouts and the x / y boundary kinds
the entry point accepts, and after the inflow was changed (the stored
deviations then keep the creation-time reference velocity).  Two calls in a
row, on two different states, check that nothing from one call leaks into
the next through the shared array.
"""
import struct

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1806_09403_gb300 import _build  # noqa: E402
from paper_1806_09403_gb300 import btdf as B  # noqa: E402

CD_TOL = 1e-4          # relative tolerance of body forces in the parity tests
FB_TOL = 2e-5          # per-marker F_b tolerance of the parity tests, times U

BOUNDARIES = {
    "inlet_freeslip": (W.BCX_INOUT, W.BCY_FREESLIP),
    "periodic": (W.BCX_PERIODIC, W.BCY_PERIODIC),
    "periodic_noslip": (W.BCX_PERIODIC, W.BCY_NOSLIP),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def compare_two_calls(case, lat, cfg, steps=(37, 11), inflow=None):
    """Two calls in a row, each on the state the context holds, against the
    context's own next step."""
    body = case.bodies[0]
    n = len(body.X)
    stream = torch.cuda.current_stream().cuda_stream
    fb = torch.full((2 * n,), float("nan"), dtype=torch.float32, device="cuda")
    for k in steps:
        lat.step(k)
        blob = lat.save_state()
        pull = struct.unpack_from("<i", blob, 24)[0] == 0     # post-collision state
        u_ref = struct.unpack_from("<d", blob, 40)[0]
        assert u_ref == case.u_in
        pops = torch.frombuffer(bytearray(blob[B.STATE_HEADER_BYTES:]), dtype=torch.uint8).cuda()
        torch.cuda.synchronize()
        rc, (Fx, Fy) = B.btdf_ib_forces_static(cfg, pops.data_ptr(), pull, body.X, body.Y,
                                               body.ds, body.Ubx, body.Uby, fb_ptr=fb.data_ptr(),
                                               stream=stream, u_ref=u_ref)
        assert rc == B.BTDF_OK
        got = fb.cpu().numpy().reshape(n, 2)
        # the regular path: the context's next step runs its IB stage on the same state
        first = lat.steps
        lat.step(1)
        ref = lat.markers(0)
        rx, ry = lat.forces(0, first, 1)
        assert np.abs(got[:, 0] - ref["Fbx"]).max() <= FB_TOL * case.u_in
        assert np.abs(got[:, 1] - ref["Fby"]).max() <= FB_TOL * case.u_in
        scale = max(abs(rx[0]), abs(ry[0]))
        assert abs(Fx - rx[0]) <= CD_TOL * scale
        assert abs(Fy - ry[0]) <= CD_TOL * scale
    return pops, pull, fb


@pytest.mark.parametrize("storage", [B.BTDF_F32, B.BTDF_F16DEV, B.BTDF_BF16DEV])
@pytest.mark.parametrize("layout", [B.LAYOUT_ROWS, B.LAYOUT_PLANES])
@pytest.mark.parametrize("bc", list(BOUNDARIES))
def test_static_ib_forces_match_context(storage, layout, bc):
    case = W.small_cylinder(delta=3, seed=21)
    case.bc_x, case.bc_y = BOUNDARIES[bc]
    lat = B.Lattice.from_case(case, storage=storage, layout=layout)
    compare_two_calls(case, lat, lat.cfg)


@pytest.mark.parametrize("delta", [2, 4, 5])
def test_static_ib_forces_other_deltas(delta):
    case = W.small_cylinder(delta=delta, seed=22)
    lat = B.Lattice.from_case(case)
    compare_two_calls(case, lat, lat.cfg)


def test_static_after_inflow_change():
    """After btdf_set_inflow the context's deviations stay relative to the
    creation-time velocity (the checkpoint header records it) while the
    inlet rule extrapolates to the new speed: the call takes both."""
    case = W.small_cylinder(delta=3, seed=23)
    lat = B.Lattice.from_case(case)
    lat.step(20)
    lat.set_inflow(0.04)
    cfg = B.btdf_config.from_buffer_copy(lat.cfg)
    cfg.u_in = 0.04
    pops, pull, fb = compare_two_calls(case, lat, cfg, steps=(17, 5))
    # the new speed taken as the reference velocity reads another state
    body = case.bodies[0]
    rc, (Fx, _) = B.btdf_ib_forces_static(cfg, pops.data_ptr(), pull, body.X, body.Y, body.ds,
                                          fb_ptr=fb.data_ptr(), u_ref=0.04,
                                          stream=torch.cuda.current_stream().cuda_stream)
    assert rc == B.BTDF_OK
    rx, _ = lat.forces(0, lat.steps - 1, 1)
    assert abs(Fx - rx[0]) > 1e-2 * abs(rx[0])


def test_static_rejects_too_many_markers():
    cfg = B.btdf_config_default()
    n = B.STATIC_MAX_MARKERS + 1
    X = np.full(n, 10.0)
    rc, _ = B.btdf_ib_forces_static(cfg, 1, False, X, X, 1.0, fb_ptr=1)
    assert rc == B.BTDF_EINVAL
