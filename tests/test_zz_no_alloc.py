"""The allocation-free binning entry point (gs_bin_atoms_static), for callers
that cannot let the library allocate device memory.  Checked through the C
ABI against the allocating entry point (gs_bin_atoms) on two calls in a row
with different inputs, so a call cannot lean on what the previous one left
in the shared scratch array.  Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

gs = pytest.importorskip("paper_1611_03474_gb300")
torch = pytest.importorskip("torch")


def _case(seed, n, cell, dims):
    rng = np.random.default_rng(seed)
    origin = np.array([-40.0, -35.0, -30.0])
    xyz = origin + rng.uniform(0, 1, (n, 3)) * (np.array(dims) * cell)
    return xyz, origin, np.array(dims, dtype=np.int64)


def test_static_binning_matches_allocating_entry_point():
    assert torch.cuda.is_available()
    cases = [(_case(21, 200003, 1.7, (40, 45, 50)), 1.7), (_case(22, 777, 3.1, (9, 7, 5)), 3.1),
             (_case(23, 5000, 2.0, (1, 1, 1)), 2.0)]
    for (xyz, origin, dims), cell in cases:
        ref_cs, ref_pm = gs.gs_bin_atoms(xyz, cell, origin, dims)
        ncell = int(np.prod(dims))
        x_d = torch.from_numpy(xyz).cuda()
        cs = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
        pm = torch.full((len(xyz),), -7, dtype=torch.int32, device="cuda")
        gs.gs_bin_atoms_static(x_d, cell, origin, dims, cs, pm)
        torch.cuda.synchronize()
        assert np.array_equal(cs.cpu().numpy(), ref_cs)
        assert np.array_equal(pm.cpu().numpy(), ref_pm)


def test_static_binning_rejects_oversized_requests():
    x_d = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    cs = torch.zeros(2, dtype=torch.int32, device="cuda")
    pm = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(gs.GsError) as e:
        gs.gs_bin_atoms_static(x_d, 1.0, np.zeros(3), np.array([2048, 1024, 1]), cs, pm)
    assert e.value.code == -1
    with pytest.raises(gs.GsError) as e:
        gs.gs_bin_atoms_static(np.zeros((4, 3)), 1.0, np.zeros(3), np.array([1, 1, 1]), cs, pm)
    assert e.value.code == -1


def test_static_binning_rejects_wrong_buffers():
    """Wrong dtype, short buffers and host tensors are refused before any GPU
    work (GsError, code -1)."""
    n, dims = 100, np.array([4, 4, 4])
    x_d = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    ok_cs = torch.zeros(65, dtype=torch.int32, device="cuda")
    ok_pm = torch.zeros(n, dtype=torch.int32, device="cuda")
    bad = [(x_d.float(), ok_cs, ok_pm), (x_d, ok_cs[:64], ok_pm), (x_d, ok_cs, ok_pm[:99]),
           (x_d, ok_cs.long(), ok_pm), (x_d.cpu(), ok_cs, ok_pm), (x_d, ok_cs, ok_pm.cpu())]
    for a, cs, pm in bad:
        with pytest.raises(gs.GsError) as e:
            gs.gs_bin_atoms_static(a, 1.0, np.zeros(3), dims, cs, pm)
        assert e.value.code == -1
