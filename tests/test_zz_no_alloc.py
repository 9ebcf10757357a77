"""The allocation-free CIC deposit (pm_cic_deposit_noalloc) for callers that
cannot let a library allocate device memory (caller-owned memory pools,
pipelines that cannot take cudaMalloc's synchronisation).

Called through the C-ABI on device arrays, several times in a row with
different particle loads and mesh sizes up to the scratch array's limit of
128^3 cells (the shared static scratch keeps the previous call's contents,
so each later result also checks that every call clears it), and compared
with the allocating entry point pm_cic_deposit (1e-12) and with the oracle's
FP64 CIC density (within the fixed-point sums' bound).  Collected last, so
that a run that stops at the first failure has run everything else."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2110_00566_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2110_00566_gb300 import binding
    return binding


def test_noalloc_deposit_matches_allocating_deposit(lib):
    L = lib.lib()
    ctx = lib.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    try:
        for seed, ng, nps in ((11, 64, 32), (12, 96, 48), (13, 128, 64), (14, 128, 128), (15, 32, 16)):
            pos_h, _ = inputs.zeldovich(nps, ng, 2.0 * ng, inputs.pk_cutoff(), 1.0, seed=seed)
            pos = torch.from_numpy(pos_h).to(dev)
            ref = torch.empty((ng,) * 3, dtype=torch.float64, device=dev)
            lib.pm_cic_deposit(ctx, ng, pos, ref)
            out = torch.full((ng,) * 3, 7.0, dtype=torch.float64, device=dev)
            rc = L.pm_cic_deposit_noalloc(ng, C.c_void_p(pos.data_ptr()), pos.shape[0],
                                          C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
            assert rc == lib.MG_OK
            torch.cuda.synchronize(dev)
            diff = (out - ref).abs().max().item()
            assert diff <= 1e-12, diff
            assert abs(out.mean().item()) < 1e-12
            # against the oracle: each CIC weight is summed as a 32.32
            # fixed-point number (at most 2^-33 from the FP64 weight), the
            # bound of the allocating deposit's own parity test
            orc, _ = oracle.cic_deposit(pos_h, ng, nps)
            scale = float(ng) ** 3 / pos_h.shape[0]
            assert np.abs(out.cpu().numpy() - orc).max() < 1e-8 * scale
    finally:
        ctx.close()


def test_noalloc_rejects_meshes_beyond_its_scratch(lib):
    L = lib.lib()
    dev = torch.device("cuda", 0)
    pos = torch.zeros((8, 3), dtype=torch.float32, device=dev)
    out = torch.zeros((130,) * 3, dtype=torch.float64, device=dev)
    rc = L.pm_cic_deposit_noalloc(130, C.c_void_p(pos.data_ptr()), 8, C.c_void_p(out.data_ptr()), None)
    assert rc == lib.MG_ERR_ARG
    host = np.zeros((16,) * 3)
    rc = L.pm_cic_deposit_noalloc(16, C.c_void_p(pos.data_ptr()), 8, C.c_void_p(host.ctypes.data), None)
    assert rc == lib.MG_ERR_ARG
