"""The no-allocation reduction entry point (collected last on purpose).

Callers whose allocator owns the whole GPU, or that cannot afford the
synchronisation an allocation may cause, use msp_reduce_lattice_noalloc():
the same lattice build and LLL kernels as the context path, with scratch in
a static device array.  Its output must equal the context path's reduced
basis exactly (integer results), on two calls in a row that share the array.
"""
import numpy as np
import pytest

from paper_2508_08702_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2508_08702_gb300 import build
    build.build()


def test_noalloc_reduction_equals_context_reduction_twice():
    from paper_2508_08702_gb300 import msp as M
    insts = [I.batch_m4_7(4)[3], I.single_m3()[0], I.batch_m4_7(4)[3]]   # m=7, m=3, m=7 again
    for inst in insts:
        m, n = inst.m, inst.n
        A = torch.from_numpy(inst.A).cuda()
        d = torch.from_numpy(inst.d).cuda()
        out = torch.full(((n + 1) * (m + n + 1),), -7, dtype=torch.int64, device="cuda")
        st = M.msp_reduce_lattice_noalloc(A, d, out)
        assert st == M.MSP_OK
        ctx = M.Context()
        pk = I.pack([inst])
        ctx.msp_build_lattice(pk.dims, pk.A, pk.d)
        ctx.msp_reduce()
        ref = ctx.msp_export_reduced(0)
        ctx.close()
        assert np.array_equal(out.cpu().numpy().reshape(n + 1, m + n + 1), ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2508_08702_gb300 import msp as M
    A = torch.zeros((4, 128), dtype=torch.int32, device="cuda")
    d = torch.zeros(4, dtype=torch.int64, device="cuda")
    out = torch.zeros(129 * 133, dtype=torch.int64, device="cuda")
    assert M.msp_reduce_lattice_noalloc(A, d, out) == M.MSP_EINVAL
