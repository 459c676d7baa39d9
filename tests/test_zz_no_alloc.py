"""lb_reduce_fields_noalloc: the mass / residual reduction for callers that cannot
allocate device memory (a host application that fixes the memory budget, or an
allocator owned by another framework). It keeps its partial sums and the previous
velocity in a fixed array inside the library, so the caller passes only its input
fields and a host output.

This file sorts last so that, in a run that stops at the first failure, every other
test has already run."""
import numpy as np
import pytest

from lbinputs import couette


def test_rejects_sizes_beyond_its_scratch_array():
    import paper_1007_4895_gb300 as lb
    fake = 256   # never dereferenced: the size check comes first
    for n in (0, lb.LB_NOALLOC_MAX_NODES + 1):
        with pytest.raises(lb.LBError) as e:
            lb.lb_reduce_fields_noalloc(fake, fake, fake, n)
        assert e.value.code == lb.LB_ERR_INVALID
        assert "scratch" in lb.lb_last_error()


@pytest.mark.gpu
def test_matches_lb_reductions_on_two_calls_in_a_row():
    import torch

    import paper_1007_4895_gb300 as lb
    w = couette(nx=300, ny=37, rows=5, kn=0.1, u_wall_lat=0.05)
    lat = lb.Lattice.from_workload(w, store="f64")
    mask = 0b111   # rho, ux, uy
    fields = torch.empty((3, w.ny, w.nx), device="cuda", dtype=torch.float64)
    stream = torch.cuda.current_stream().cuda_stream
    n = w.nx * w.ny
    assert n <= lb.LB_NOALLOC_MAX_NODES
    tol = 1e-10   # the FP64 parity tolerance of the other tests

    lat.step(40)
    ref1 = lat.reductions()
    lat.moments_into(fields, mask)
    got1 = lb.lb_reduce_fields_noalloc(fields[0].data_ptr(), fields[1].data_ptr(), fields[2].data_ptr(), n,
                                       restart=True, stream=stream)
    np.testing.assert_allclose(got1[0], ref1["mass"], rtol=tol)
    np.testing.assert_allclose(got1[1], ref1["residual"], rtol=tol)
    assert got1[2] == 0 and got1[3] == n

    lat.step(25)
    ref2 = lat.reductions()
    lat.moments_into(fields, mask)
    got2 = lb.lb_reduce_fields_noalloc(fields[0].data_ptr(), fields[1].data_ptr(), fields[2].data_ptr(), n,
                                       stream=stream)
    np.testing.assert_allclose(got2[0], ref2["mass"], rtol=tol)
    np.testing.assert_allclose(got2[1], ref2["residual"], rtol=tol)
    assert 0 < got2[1] < 1 and got2[2] == 0


@pytest.mark.gpu
def test_a_non_finite_node_is_reported_and_its_velocity_kept():
    """A node that is non-finite on one call is counted and makes the call fail with
    LB_ERR_DIVERGED; its velocity is still kept, so the next call (without restart)
    compares with it and gives a non-finite residual; a restart clears that."""
    import torch

    import paper_1007_4895_gb300 as lb
    n = 4096
    g = torch.Generator(device="cpu").manual_seed(3)
    rho = (1.0 + 0.01 * torch.rand(n, generator=g, dtype=torch.float64)).cuda()
    ux = (0.01 * torch.rand(n, generator=g, dtype=torch.float64)).cuda()
    uy = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    args = (rho.data_ptr(), ux.data_ptr(), uy.data_ptr(), n)
    ok = lb.lb_reduce_fields_noalloc(*args, restart=True, stream=stream)
    assert ok[2] == 0
    ux[17] = float("nan")
    with pytest.raises(lb.LBError) as e:
        lb.lb_reduce_fields_noalloc(*args, stream=stream)
    assert e.value.code == lb.LB_ERR_DIVERGED
    ux[17] = 0.005
    again = lb.lb_reduce_fields_noalloc(*args, stream=stream)
    assert again[2] == 0 and not np.isfinite(again[1])
    fresh = lb.lb_reduce_fields_noalloc(*args, restart=True, stream=stream)
    assert fresh[2] == 0 and np.isfinite(fresh[1])
    np.testing.assert_allclose(fresh[0], rho.sum().item(), rtol=1e-12)
