"""The allocation-free dot product (fe_dot_noalloc) against the library's existing reductions.

fe_dot_noalloc serves callers that may not allocate device memory (for
example a host application that owns the whole device memory budget, or a
latency-critical loop where cudaMalloc's implicit synchronisation is not
allowed); its scratch is a static device array of the library.  This file is
collected last so that a failure here cannot hide the other tests.  It checks,
through the C ABI, that two calls in a row reproduce the objective J =
(u - u_d)^T M (u - u_d) computed by the existing entry point fe_objective,
within the FP64 tolerance the other parity tests use.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08012_gb300 import build
    build.build()
    import paper_2104_08012_gb300 as fe
    fe.load()
    return fe


def test_dot_noalloc_matches_objective(fe):
    import fe_inputs as I
    with fe.Hierarchy(4, 1, 2) as h:  # P2 on 8^3: 4913 dofs, spans several partial sums
        kappa = I.grf_kappa(h.cell_centroids(), seed=31)
        h.set_coefficient(torch.from_numpy(kappa).cuda())
        n = h.n_dofs()
        u = torch.from_numpy(I.random_vector(n, 41)).cuda()
        ud = torch.from_numpy(I.target_field(h.dof_coordinates())).cuda()
        J_ref = h.objective(u, ud)  # existing entry point
        e = u - ud
        Me = torch.empty_like(e)
        h.apply_mass(e, Me)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        vals = []
        for _ in range(2):  # two calls in a row share (and must clear) the static scratch
            fe.fe_dot_noalloc(e, Me, out=out)
            torch.cuda.synchronize()
            vals.append(out.item())
        vals.append(fe.fe_dot_noalloc(e, Me))  # host output
        for v in vals:
            assert abs(v - J_ref) <= 1e-13 * abs(J_ref), (v, J_ref)
        assert vals[0] == vals[1] == vals[2]


def test_dot_noalloc_large_and_limits(fe):
    n = 5_000_003  # ragged tail, many partial sums
    g = torch.Generator(device="cpu").manual_seed(3)
    x = torch.rand(n, dtype=torch.float64, generator=g).cuda()
    y = torch.rand(n, dtype=torch.float64, generator=g).cuda()
    a = fe.fe_dot_noalloc(x, y)
    b = fe.fe_dot_noalloc(x, y)
    ref = float(np.dot(x.cpu().numpy(), y.cpu().numpy()))
    assert a == b and abs(a - ref) <= 1e-13 * abs(ref)
    assert fe.fe_dot_noalloc(x, y, n=0) == 0.0
    with pytest.raises(fe.FeError) as err:
        fe.fe_dot_noalloc(x, y, n=67_108_865)
    assert err.value.code == fe.FE_ERR_ARG
    with pytest.raises(fe.FeError) as err:
        fe.fe_dot_noalloc(x.cpu().numpy(), y)
    assert err.value.code == fe.FE_ERR_ARG


def test_dot_noalloc_rejects_bad_buffers(fe):
    """Buffers that do not hold what the call reads or writes are rejected before any launch."""
    x = torch.rand(64, dtype=torch.float64, device="cuda")
    y = torch.rand(64, dtype=torch.float64, device="cuda")
    launches = fe.fe_kernel_launches()
    bad = [
        dict(x=x.float(), y=y.float()),                               # float32 vectors
        dict(x=x, y=y, n=65),                                         # n beyond the vectors
        dict(x=x, y=y[:32], n=64),                                    # n beyond y
        dict(x=x, y=y, out=torch.zeros(1, dtype=torch.float32, device="cuda")),  # float32 out
        dict(x=x, y=y, out=torch.zeros(0, dtype=torch.float64, device="cuda")),  # empty out
        dict(x=x[::2], y=y[::2]),                                     # strided views
        dict(x=x.cpu(), y=y),                                         # x on the host
    ]
    for kw in bad:
        with pytest.raises(fe.FeError) as err:
            fe.fe_dot_noalloc(**kw)
        assert err.value.code == fe.FE_ERR_ARG, kw
    assert fe.fe_kernel_launches() == launches


def test_dot_noalloc_allocates_nothing(fe):
    """The property the entry point exists for: after the first call on the device (which looks up the
    static array's address), further calls change neither torch's allocations nor the device's free memory."""
    n = 300_001
    x = torch.rand(n, dtype=torch.float64, device="cuda")
    y = torch.rand(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    fe.fe_dot_noalloc(x, y, out=out)
    fe.fe_dot_noalloc(x, y)
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    vals = []
    for _ in range(4):
        fe.fe_dot_noalloc(x, y, out=out)
        torch.cuda.synchronize()
        vals.append(out.item())
        vals.append(fe.fe_dot_noalloc(x, y))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0
    assert len(set(vals)) == 1
