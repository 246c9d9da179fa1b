"""The C-ABI library loads, exports every symbol include/btdf.h declares, and
rejects invalid configurations on the host before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1806_09403_gb300 import _build
from paper_1806_09403_gb300 import btdf as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "btdf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(btdf_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    L = ctypes.CDLL(_build.LIB)
    decl = declared_symbols()
    assert len(decl) >= 20
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(B.EXPORTS) == decl


def test_config_struct_size_matches():
    # 2 int32 + 2 double + 6 int32 + 2 double + 2 int32, no padding holes
    assert ctypes.sizeof(B.btdf_config) == 72


def test_variant_count_matches_header():
    src = open(os.path.join(ROOT, "include", "btdf.h")).read()
    m = re.search(r"#define BTDF_VARIANT_COUNT (\d+)", src)
    assert m and int(m.group(1)) == B.VARIANT_COUNT
    # every variant the header documents under btdf_tune, 0 .. count - 1
    doc = src[src.index("Variant of the fused collide-stream kernel"):src.index("int btdf_tune(")]
    listed = sorted({int(v) for v in re.findall(r"\n \*\s+(\d+) ", doc)})
    assert listed == list(range(B.VARIANT_COUNT))


def test_version_and_status_strings():
    assert B.btdf_version() >= 1
    for rc in (0, -1, -2, -3, -4, -5, -6):
        assert B.btdf_status_string(rc) != "unknown status"


@pytest.mark.parametrize("field,value", [
    ("tau", 0.5), ("tau", float("nan")), ("nx", 3), ("ny", 0), ("delta", 1), ("delta", 6),
    ("nf", 0), ("nf", 65), ("storage", 3), ("bc_x", 4), ("bc_y", 3), ("history_len", 0),
    ("u_in", float("inf")), ("u_in", 0.6), ("gx", float("nan")), ("layout", 2),
])
def test_invalid_config_rejected_on_host(field, value):
    cfg = B.btdf_config_default()
    setattr(cfg, field, value)
    rc, ctx = B.btdf_create(cfg)
    assert rc == B.BTDF_EINVAL
    assert not ctx


def test_lattice_beyond_32bit_offsets_rejected_on_host():
    """Element offsets inside the kernels are 32-bit: 9 x nxp x ny must stay
    below 2^32 (nxp = nx rounded up to 32).  32768 x 14563 is the largest
    lattice of that width; one more row is refused before any device call."""
    cfg = B.btdf_config_default()
    cfg.nx, cfg.ny = 32768, 14564
    assert 9 * 32768 * 14564 >= 2 ** 32 > 9 * 32768 * 14563
    rc, ctx = B.btdf_create(cfg)
    assert rc == B.BTDF_EINVAL and not ctx


def test_null_arguments_rejected():
    L = B.lib()
    assert L.btdf_create(None, None, None) == B.BTDF_EINVAL
    assert L.btdf_destroy(None) == B.BTDF_EINVAL
    assert L.btdf_step(None, 1) == B.BTDF_EINVAL
    assert L.btdf_step_count(None) == -1


def test_no_gpu_reports_cuda_error_not_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    cfg = B.btdf_config_default()
    rc, ctx = B.btdf_create(cfg)
    assert rc == B.BTDF_ECUDA and not ctx


def test_batch_rejects_mixed_delta_and_mdf():
    import ctypes as C
    cfgs = (B.btdf_config * 2)(B.btdf_config_default(), B.btdf_config_default())
    cfgs[1].delta = 4
    out = C.c_void_p()
    assert B.lib().btdf_batch_create(cfgs, 2, None, C.byref(out)) == B.BTDF_EINVAL
    cfgs[1].delta = 3
    cfgs[1].nf = 2
    assert B.lib().btdf_batch_create(cfgs, 2, None, C.byref(out)) == B.BTDF_EINVAL
    assert B.lib().btdf_batch_create(cfgs, 0, None, C.byref(out)) == B.BTDF_EINVAL


@pytest.mark.parametrize("storage,pops,fb", [
    (0, 16, 4),      # F_b not 8-byte aligned
    (0, 18, 16),     # FP32 populations not 4-byte aligned
    (1, 17, 16),     # FP16 populations not 2-byte aligned
    (2, 33, 64),     # BF16 populations not 2-byte aligned
])
def test_static_rejects_misaligned_pointers(storage, pops, fb):
    """btdf_ib_forces_static refuses misaligned device pointers with EINVAL
    before any device work (the pointer values here are never dereferenced)."""
    cfg = B.btdf_config_default()
    cfg.storage = storage
    X = np.full(10, 10.0)
    rc, _ = B.btdf_ib_forces_static(cfg, pops, False, X, X, 1.0, fb_ptr=fb)
    assert rc == B.BTDF_EINVAL


@pytest.mark.parametrize("u_ref", [float("nan"), 0.5, -0.7])
def test_static_rejects_bad_reference_velocity(u_ref):
    cfg = B.btdf_config_default()
    X = np.full(10, 10.0)
    rc, _ = B.btdf_ib_forces_static(cfg, 16, False, X, X, 1.0, fb_ptr=16, u_ref=u_ref)
    assert rc == B.BTDF_EINVAL
