"""dg_conserved_static: the conserved sums computed without allocating device memory.

Some callers cannot call cudaMalloc when they need these sums (a host code whose
GPU memory is all reserved for its own pool, or a loop that must not take the
synchronisation an allocation can cause).  dg_conserved_static serves them with a
fixed scratch array inside libdg.so.  These tests call it through the C ABI and
compare it with dg_conserved, which allocates its scratch per handle.  The file
is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1805_01443_gb300 import dg, inputs


def _spacing(cfg):
    m = cfg["mesh"]
    return (m["x1"] - m["x0"]) / m["nx"], (m["y1"] - m["y0"]) / m["ny"]


@pytest.mark.gpu
def test_conserved_static_matches_dg_conserved_on_two_calls_in_a_row():
    import torch

    L = dg.lib()
    cases = []
    # a larger mesh first, then a smaller one: the second call must not see the
    # first call's leftover partial sums in the shared scratch array
    for cfg in [inputs.disc_planet(96, 3), inputs.density_wave(20, 2)]:
        with dg.Disc(cfg) as d:
            d.step(2)
            ref = d.conserved()
            host = d.fetch()
        dev = torch.from_numpy(host).to("cuda")
        out = torch.full((host.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        cases.append((cfg, ref, dev, out))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    for cfg, ref, dev, out in cases:
        nv, nmodes, ny, nx = dev.shape
        dx, dy = _spacing(cfg)
        rc = L.dg_conserved_static(ctypes.c_void_p(dev.data_ptr()), nv, nmodes, nx, ny, dx, dy,
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == dg.DG_OK
    torch.cuda.synchronize()
    for cfg, ref, dev, out in cases:
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.gpu
def test_conserved_static_allocates_nothing_after_the_first_call():
    """The property the call exists for: once a first call has loaded the
    library's scratch array on the device, a call changes neither the device's
    free memory (cudaMemGetInfo) nor PyTorch's allocator counters."""
    import torch

    L = dg.lib()
    cfg = inputs.disc_planet(64, 2)
    with dg.Disc(cfg) as d:
        d.step(1)
        ref = d.conserved()
        host = d.fetch()
    dev = torch.from_numpy(host).to("cuda")
    out = torch.zeros(host.shape[0], dtype=torch.float64, device="cuda")
    nv, nmodes, ny, nx = dev.shape
    dx, dy = _spacing(cfg)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (ctypes.c_void_p(dev.data_ptr()), nv, nmodes, nx, ny, dx, dy, ctypes.c_void_p(out.data_ptr()),
            stream)
    assert L.dg_conserved_static(*args) == dg.DG_OK  # the warm-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    allocated0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert L.dg_conserved_static(*args) == dg.DG_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == allocated0
    for key in ("allocation.all.allocated", "segment.all.allocated"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_conserved_static_rejects_bad_sizes_before_any_launch():
    """Sizes above DG_STATIC_MAX_ELEMENTS and null pointers are refused on the host
    (no CUDA call is made, so this runs without a GPU)."""
    L = dg.lib()
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check fails first
    assert L.dg_conserved_static(fake, 3, 25, 1025, 1024, 1.0, 1.0, fake, None) == dg.DG_ERR_ARG
    assert L.dg_conserved_static(None, 3, 25, 8, 8, 1.0, 1.0, fake, None) == dg.DG_ERR_ARG
    assert L.dg_conserved_static(fake, 5, 25, 8, 8, 1.0, 1.0, fake, None) == dg.DG_ERR_ARG
    assert L.dg_conserved_static(fake, 3, 25, 8, 8, 0.0, 1.0, fake, None) == dg.DG_ERR_ARG


def test_conserved_static_refuses_host_memory():
    """Host arrays (here numpy's) are refused with DG_ERR_ARG before any launch,
    with a GPU (the pointer is not device memory) and without one (there is no
    current device)."""
    L = dg.lib()
    coeffs = np.zeros((3, 9, 8, 8))
    out = np.zeros(3)
    rc = L.dg_conserved_static(coeffs.ctypes.data_as(ctypes.c_void_p), 3, 9, 8, 8, 1.0, 1.0,
                               out.ctypes.data_as(ctypes.c_void_p), None)
    assert rc == dg.DG_ERR_ARG
    assert b"dg_conserved_static" in L.dg_last_error(None)
    assert np.all(out == 0.0)
