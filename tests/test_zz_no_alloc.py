"""The IB force stage for callers that cannot allocate device memory.

Code that runs inside another framework's memory budget, code issued while a
CUDA stream is being captured into a graph, and real-time loops cannot call
cudaMalloc.  They use btdf_ib_forces_static, whose scratch is a fixed
file-scope device array.  Here it must agree with the regular path: a
context's own IB stage applied to the same populations.  Two calls in a row,
on two different states, check that nothing from one call leaks into the
next through the shared array.
"""
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


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


@pytest.mark.parametrize("delta", [3, 5])
def test_static_ib_forces_match_context(delta):
    case = W.small_cylinder(delta=delta, seed=21)
    body = case.bodies[0]
    n = len(body.X)
    lat = B.Lattice.from_case(case)
    stream = torch.cuda.current_stream().cuda_stream
    fb = torch.full((2 * n,), float("nan"), dtype=torch.float32, device="cuda")
    for steps in (37, 11):                       # two calls in a row
        lat.step(steps)
        blob = lat.save_state()
        pull = int.from_bytes(blob[24:28], "little") == 0     # post-collision state
        pops = torch.frombuffer(bytearray(blob[B.STATE_HEADER_BYTES:]), dtype=torch.uint8).cuda()
        torch.cuda.synchronize()
        rc, (Fx, Fy) = B.btdf_ib_forces_static(lat.cfg, pops.data_ptr(), pull, body.X, body.Y,
                                               body.ds, body.Ubx, body.Uby, fb_ptr=fb.data_ptr(),
                                               stream=stream)
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


def test_static_rejects_too_many_markers():
    cfg = B.btdf_config_default()
    n = B.STATIC_MAX_MARKERS + 1
    X = np.full(n, 10.0)
    rc, _ = B.btdf_ib_forces_static(cfg, 1, False, X, X, 1.0, fb_ptr=1)
    assert rc == B.BTDF_EINVAL
