"""The C ABI library builds, loads and exports every function include/dg.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

import pytest

from paper_1805_01443_gb300 import build as dgbuild
from paper_1805_01443_gb300 import dg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    dgbuild.build()
    return dg.lib()


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for required in ["dg_init", "dg_step", "dg_torque", "dg_fetch", "dg_set_state",
                     "dg_torque_series", "dg_get_time", "dg_set_stream", "dg_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(dg.EXPORTED)


def test_argument_validation_without_gpu(L):
    """Invalid arguments are rejected on the host before any CUDA call."""
    from paper_1805_01443_gb300 import inputs
    cfg = inputs.disc_small(8, 2)
    with pytest.raises(dg.DgError) as e:
        bad = dict(cfg, order=7)
        dg.dg_workspace_bytes(bad)
    assert e.value.code == dg.DG_ERR_UNSUPPORTED
    bad = inputs.disc_small(8, 2)
    bad["mesh"]["nx"] = 0
    with pytest.raises(dg.DgError) as e:
        dg.dg_workspace_bytes(bad)
    assert e.value.code == dg.DG_ERR_ARG
    bad = inputs.disc_small(8, 2)
    bad["disc"]["r_soft"] = 0.0
    with pytest.raises(dg.DgError) as e:
        dg.dg_workspace_bytes(bad)
    assert e.value.code == dg.DG_ERR_ARG
    # the paper's own disc (ic 6) needs the adiabatic EOS and the star
    assert dg.dg_workspace_bytes(inputs.paper_disc(16, 2)) > 0
    bad = inputs.paper_disc(16, 2)
    bad["eos"]["kind"] = 0
    with pytest.raises(dg.DgError) as e:
        dg.dg_workspace_bytes(bad)
    assert e.value.code == dg.DG_ERR_ARG
    bad = inputs.paper_disc(16, 2)
    bad["disc"]["star"] = 0
    with pytest.raises(dg.DgError) as e:
        dg.dg_workspace_bytes(bad)
    assert e.value.code == dg.DG_ERR_ARG
    assert dg.dg_workspace_bytes(cfg) > 0


def test_workspace_size_scales_with_mesh(L):
    from paper_1805_01443_gb300 import inputs
    a = dg.dg_workspace_bytes(inputs.disc_planet(64, 4))
    b = dg.dg_workspace_bytes(inputs.disc_planet(128, 4))
    assert 3.5 < b / a < 4.5


def _bad(edit):
    from paper_1805_01443_gb300 import inputs
    cfg = inputs.disc_small(8, 2)
    edit(cfg)
    return cfg


def _set(section, **kw):
    return lambda c: c[section].update(kw)


@pytest.mark.parametrize("edit,code", [
    (_set("mesh", nx=70000), dg.DG_ERR_ARG),                         # side outside 1..65535
    (_set("mesh", nx=20000, ny=20000), dg.DG_ERR_ARG),               # more than 2^28 elements
    (_set("mesh", x1=-3.0), dg.DG_ERR_ARG),                          # empty box
    (_set("mesh", bc=4), dg.DG_ERR_ARG),
    (lambda c: c.update(order=0), dg.DG_ERR_UNSUPPORTED),
    (_set("eos", kind=3), dg.DG_ERR_UNSUPPORTED),
    (_set("eos", kind=1, gamma=1.0), dg.DG_ERR_ARG),
    (_set("disc", ic=7), dg.DG_ERR_UNSUPPORTED),
    (_set("disc", ic=4), dg.DG_ERR_ARG),                             # vortex needs the adiabatic EOS
    (lambda c: (c["eos"].update(kind=1), c["disc"].update(ic=3, ring_p=0.0)), dg.DG_ERR_ARG),
    (_set("disc", limiter=3), dg.DG_ERR_ARG),
    (_set("disc", positivity=1, rk=2), dg.DG_ERR_UNSUPPORTED),       # limiters need SSP(3,3)
    (_set("disc", limiter=1, tvb_m=-1.0), dg.DG_ERR_ARG),
    (_set("disc", rk=6), dg.DG_ERR_UNSUPPORTED),
    (_set("disc", rk=4, prec=1), dg.DG_ERR_UNSUPPORTED),             # RK(4,5) in the FP64 form only
    (_set("disc", prec=2), dg.DG_ERR_UNSUPPORTED),                   # only FP64 and the FP32 form
    (lambda c: (c["eos"].update(kind=1), c["disc"].update(prec=1)), dg.DG_ERR_UNSUPPORTED),
    (_set("disc", cfl=0.0), dg.DG_ERR_ARG),
])
def test_every_validation_rule_returns_its_documented_code(L, edit, code):
    """Each host-side check of dg_init (run here through dg_workspace_bytes,
    before any CUDA call) rejects with the code include/dg.h documents."""
    with pytest.raises(dg.DgError) as e:
        dg.dg_workspace_bytes(_bad(edit))
    assert e.value.code == code


def test_no_cpu_fallback_without_a_device(L):
    """Without a CUDA device the binding raises instead of computing anything:
    through PyTorch's allocator, and through dg_init's own allocation."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_1805_01443_gb300 import inputs
    cfg = inputs.disc_small(8, 2)
    with pytest.raises(RuntimeError, match="no CPU path"):
        dg.Disc(cfg)
    with pytest.raises(dg.DgError) as e:
        dg.Disc(cfg, torch_memory=False)
    assert e.value.code in (dg.DG_ERR_NOMEM, dg.DG_ERR_CUDA)


def test_init_ex_refuses_a_host_workspace(L):
    """A caller workspace in host memory (aligned and large enough) is refused
    with DG_ERR_ARG before any allocation or launch: with a GPU it is not
    device memory, without one there is no current device."""
    import ctypes

    import numpy as np
    from paper_1805_01443_gb300 import inputs
    cfg = inputs.disc_small(8, 2)
    nbytes = dg.dg_workspace_bytes(cfg)
    raw = np.zeros(nbytes + 256, dtype=np.uint8)
    off = (-raw.ctypes.data) % 256
    ws = raw[off:off + nbytes]
    mesh, order, eos, planet, disc = dg.structs(cfg)
    h = ctypes.c_void_p()
    rc = L.dg_init_ex(ctypes.byref(h), ctypes.byref(mesh), order, ctypes.byref(eos), ctypes.byref(planet),
                      ctypes.byref(disc), ctypes.c_void_p(ws.ctypes.data), nbytes, None)
    assert rc == dg.DG_ERR_ARG
    assert not h.value
    assert b"workspace" in L.dg_last_error(None)
    assert not ws.any()


def test_binding_refuses_tensors_it_cannot_pass_on():
    """The binding hands the network calls and dg_features bare data pointers:
    a host tensor, or one of another dtype, shape or layout, is refused before
    any pointer reaches the library (host logic, no device needed)."""
    torch = pytest.importorskip("torch")
    x = torch.zeros((4, 8), dtype=torch.float32)
    with pytest.raises(ValueError, match="CUDA tensor"):
        dg._device_tensor(x, torch.float32, (4, 8), "x")
    with pytest.raises(ValueError, match="CUDA tensor"):
        dg._device_tensor(x.numpy(), torch.float32, (4, 8), "x")
