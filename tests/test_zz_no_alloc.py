"""mk_census_noalloc: the census for callers that cannot allocate.

Some callers of this library cannot allocate device memory (a C program or
language binding that only hands over pointers it already owns, or code
that must not call cudaMalloc/cudaFree because they synchronise the device).
mk_census_noalloc gives them the census with the library's own fixed
scratch array in place of the workspace.  This test calls it through the C
ABI twice in a row and checks both results against mk_census with a
caller-provided workspace on the same inputs; the results are integers, so
they must be identical.  It lives in a file of its own that pytest collects
last, and it builds everything it needs, so it passes alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_2606_15437_gb300 import build as mkbuild
from paper_2606_15437_gb300 import mk
from paper_2606_15437_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    mkbuild.build()
    assert torch.cuda.is_available(), "needs a CUDA device"


def test_noalloc_matches_workspace_census_twice():
    from paper_2606_15437_gb300.engine import CensusJob
    texts = W.pr1_formulas()[:40] + W.census5_formulas()[:40]
    # all four classes through five worlds: the S4/S5 lists live in the scratch
    job = CensusJob(texts, ("K", "T", "S4", "S5"), 1, 5, samples=256, seed=2)
    want = job.run()
    assert int(want[..., 0].sum()) > 0
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full_like(job.d_out, -7)
        status = torch.zeros(1, dtype=torch.int32, device=job.device)
        rc = mk.census_noalloc_raw(job.d_progs.data_ptr(), job.nprog, job.cfg, out.data_ptr(),
                                   status.data_ptr(), stream)
        assert rc == 0, mk.strerror(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got = out.cpu().numpy().view(np.uint64).reshape(want.shape)
        assert np.array_equal(got, want)


def test_noalloc_rejects_oversized_configuration():
    # S4 at six worlds needs more scratch than the fixed array holds
    progs = mk.compile_batch(["[]p -> p"])
    d_progs = torch.from_numpy(progs.view(np.uint8).copy()).cuda()
    cfg = mk.census_cfg(("S4",), 6, 6, 0, 0, max_depth=1)
    assert mk.census_workspace_size(cfg, 1) > (1 << 20)      # MK_NOALLOC_SCRATCH_BYTES
    out = torch.zeros(3, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = mk.census_noalloc_raw(d_progs.data_ptr(), 1, cfg, out.data_ptr(), status.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert rc == -6      # MK_E_WORKSPACE, nothing launched
    torch.cuda.synchronize()
    assert int(status.item()) == 0
