"""The allocation-free binning entry point, lj_bin_cells_static.

It serves callers that cannot allocate device memory when they need cell
lists (another allocator owns the device pool, or a real-time loop must not
hit cudaMalloc's implicit synchronisation).  Its scratch is one fixed device
array inside the library.  This test calls it through the C ABI on device
buffers the test owns, twice in a row on different inputs, and checks its
outputs against the context-based lj_bin_cells and against the oracle's stable
counting sort (integer results: equal)."""
import ctypes as C

import numpy as np
import pytest

from paper_2512_03565_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_binning_matches_context_binning(orc):
    torch = pytest.importorskip("torch")
    from paper_2512_03565_gb300 import build as B
    B.build()
    from paper_2512_03565_gb300 import ljgb as lj
    lib = lj.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    systems = [W.stratified(20000, 0.75, 31), W.slab(30000, 0.8, 0.02, 0.4, 32)]
    for s in systems:
        nc = int(np.floor(s.L / s.rc))
        ncell = nc ** 3
        assert s.n <= 65536 and ncell <= 32768
        pos_d = torch.from_numpy(s.pos.view(np.int32)).to(dev).contiguous()
        perm_d = torch.zeros(s.n, dtype=torch.int32, device=dev)
        cs_d = torch.zeros(ncell + 1, dtype=torch.int32, device=dev)
        st = lib.lj_bin_cells_static(pos_d.data_ptr(), s.n, nc, perm_d.data_ptr(), cs_d.data_ptr(),
                                     stream.cuda_stream)
        assert st == lj.LJ_OK
        torch.cuda.synchronize(dev)
        d = lj.Domain(s.L, s.rc, s.skin)
        d.set_particles(s.pos)
        d.bin_cells(lj.LJ_LC)
        perm_ref, cs_ref, nc_ref = d.cells()
        d.close()
        assert nc_ref == nc
        perm_s = perm_d.cpu().numpy().view(np.uint32)
        cs_s = cs_d.cpu().numpy().view(np.uint32)
        assert np.array_equal(perm_s, perm_ref)
        assert np.array_equal(cs_s, cs_ref)
        perm_o, cs_o = orc.bin_cells(s.pos, nc)
        assert np.array_equal(perm_s, perm_o)
        assert np.array_equal(cs_s, cs_o)
    # a third call in a row at both maxima (n = 65,536 particles, 32^3 cells)
    s = W.stratified(65536, 0.75, 33)
    pos_d = torch.from_numpy(s.pos.view(np.int32)).to(dev).contiguous()
    perm_d = torch.zeros(s.n, dtype=torch.int32, device=dev)
    cs_d = torch.zeros(32 ** 3 + 1, dtype=torch.int32, device=dev)
    assert lib.lj_bin_cells_static(pos_d.data_ptr(), s.n, 32, perm_d.data_ptr(), cs_d.data_ptr(),
                                   stream.cuda_stream) == lj.LJ_OK
    torch.cuda.synchronize(dev)
    perm_o, cs_o = orc.bin_cells(s.pos, 32)
    assert np.array_equal(perm_d.cpu().numpy().view(np.uint32), perm_o)
    assert np.array_equal(cs_d.cpu().numpy().view(np.uint32), cs_o)


def test_static_binning_rejects_oversized_inputs():
    torch = pytest.importorskip("torch")
    from paper_2512_03565_gb300 import ljgb as lj
    lib = lj.load()
    dev = torch.device("cuda", 0)
    buf = torch.zeros(3 * 16, dtype=torch.int32, device=dev)
    assert lib.lj_bin_cells_static(buf.data_ptr(), 70000, 4, buf.data_ptr(), buf.data_ptr(), None) == lj.LJ_ERR_ARG
    assert lib.lj_bin_cells_static(buf.data_ptr(), 16, 33, buf.data_ptr(), buf.data_ptr(), None) == lj.LJ_ERR_ARG
    assert lib.lj_bin_cells_static(None, 16, 4, buf.data_ptr(), buf.data_ptr(), None) == lj.LJ_ERR_ARG
