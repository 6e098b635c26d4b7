"""skel_eval_velocity_noalloc, the velocity evaluation that allocates
nothing (its partial sums live in a static device array), against the
regular skel_eval_velocity through the C ABI.  Collected last on purpose:
it must pass both alone in a fresh process and after every other test."""
import numpy as np
import pytest

import workloads as W
from gpu_util import solver

pytestmark = pytest.mark.gpu

TOL = 1e-13   # same sums, possibly split into a different number of chunks


def rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case():
    import torch
    wl = W.star1()
    s = solver(wl)
    s.factor()
    dev = torch.device("cuda")
    like = torch.zeros(1, dtype=torch.float64, device=dev)
    x = s.solve(s.point_force_rhs(wl.src_xy, wl.src_f, like=like))
    tx = torch.tensor(wl.targets[:, 0].copy(), device=dev)
    ty = torch.tensor(wl.targets[:, 1].copy(), device=dev)
    rng = np.random.default_rng(21)
    sol3 = torch.tensor(rng.standard_normal((wl.n_unknowns, 3)), device=dev)
    yield s, x, sol3, tx, ty
    s.close()


def test_noalloc_matches_regular_on_calls_in_a_row(case):
    import torch
    s, x, sol3, tx, ty = case
    nt = tx.shape[0]
    # call 1: one column at every target; call 2: three columns at a few
    # targets (a different shape reuses the same static array); call 3:
    # call 1 again, which must not see call 2's leftovers
    calls = [(x, tx, ty), (sol3, tx[:37], ty[:37]), (x, tx, ty)]
    got = []
    for sol, a, b in calls:
        ref = s.eval_velocity(sol, a, b)
        nrhs = 1 if sol.dim() == 1 else sol.shape[1]
        out = torch.full((nrhs, a.shape[0], 2), float("nan"),
                         dtype=torch.float64, device=a.device)
        u = s.eval_velocity_noalloc(sol, a, b, out=out)
        assert u.shape == ref.shape
        assert torch.isfinite(u).all()
        assert rel(u, ref) < TOL
        got.append(u.clone())
    assert nt > 37
    assert torch.equal(got[0], got[2])


def test_noalloc_rejects_sizes_beyond_its_scratch(case):
    import paper_2001_11619_gb300 as skel
    import torch
    s, x, sol3, tx, ty = case
    limit = 262144                       # 4 MiB of partial sums / 2 / 8 B
    n = limit // 3 + 1                   # n * 3 columns > limit
    m = limit // 2                       # m * 2 columns == limit
    # targets at (-0.5, 0), inside the domain and away from every curve
    bx = torch.full((m,), -0.5, dtype=torch.float64, device=tx.device)
    by = torch.zeros((m,), dtype=torch.float64, device=tx.device)
    out = torch.empty((3, n, 2), dtype=torch.float64, device=tx.device)
    with pytest.raises(skel.SkelError) as e:
        s.eval_velocity_noalloc(sol3, bx[:n], by[:n], out=out)
    assert e.value.code == -3            # SKEL_ECAPACITY
    assert "262144" in str(e.value)
    # exactly at the limit is accepted
    out2 = torch.full((2, m, 2), float("nan"), dtype=torch.float64,
                      device=tx.device)
    u = s.eval_velocity_noalloc(sol3[:, :2], bx[:m], by[:m], out=out2)
    assert u.data_ptr() == out2.data_ptr()   # written in the caller's out
    ref = s.eval_velocity(sol3[:, :2], bx[:1], by[:1])
    assert rel(u[:1], ref) < TOL
    assert torch.equal(u[-1], u[0])
    # one grid row per right-hand side: more than 65535 is refused
    many = torch.zeros((65536, x.shape[0]), dtype=torch.float64,
                       device=tx.device).t()
    outm = torch.empty((65536, 1, 2), dtype=torch.float64, device=tx.device)
    with pytest.raises(skel.SkelError) as e:
        s.eval_velocity_noalloc(many, bx[:1], by[:1], out=outm)
    assert e.value.code == -1            # SKEL_EINVAL
    assert "65535" in str(e.value)


def test_noalloc_checks_out_and_targets_before_the_call(case):
    """The kernels write ``out`` in place, so its shape, dtype, layout and
    device are checked before the call, and tx, ty must match."""
    import torch
    s, x, sol3, tx, ty = case
    nt = tx.shape[0]
    f64 = dict(dtype=torch.float64, device=tx.device)
    bad = [torch.empty((1, nt - 1, 2), **f64),               # too short
           torch.empty((1, nt, 2), dtype=torch.float32,
                       device=tx.device),                     # float32
           torch.empty((1, 2, nt), **f64).transpose(1, 2),    # strided
           torch.empty((1, nt, 2), dtype=torch.float64)]      # host
    for out in bad:
        with pytest.raises(ValueError):
            s.eval_velocity_noalloc(x, tx, ty, out=out)
    with pytest.raises(ValueError):
        s.eval_velocity_noalloc(x, tx, ty[:-1],
                                out=torch.empty((1, nt, 2), **f64))
    with pytest.raises(ValueError):
        s.eval_velocity_noalloc(x, tx.float(), ty,
                                out=torch.empty((1, nt, 2), **f64))


def test_noalloc_calls_leave_free_device_memory_unchanged(case):
    """The defining property: after the first call (which looks up the
    static array), calls of several shapes change the device's free memory
    by nothing (cudaMemGetInfo before and after)."""
    import torch
    s, x, sol3, tx, ty = case
    solT = sol3.t().contiguous()         # (nrhs, n): no copy in the binding
    outs = {k: torch.empty((k, n, 2), dtype=torch.float64, device=tx.device)
            for k, n in ((1, tx.shape[0]), (3, 37), (2, 5))}
    s.eval_velocity_noalloc(x, tx, ty, out=outs[(1)])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        s.eval_velocity_noalloc(x, tx, ty, out=outs[1])
        s.eval_velocity_noalloc(solT[:3].t(), tx[:37], ty[:37], out=outs[3])
        s.eval_velocity_noalloc(solT[:2].t(), tx[:5], ty[:5], out=outs[2])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_host_arrays(case):
    import paper_2001_11619_gb300 as skel
    s, x, sol3, tx, ty = case
    with pytest.raises(skel.SkelError) as e:
        s.eval_velocity_noalloc(x, tx.cpu().numpy(), ty.cpu().numpy(),
                                out=np.empty((1, tx.shape[0], 2)))
    assert e.value.code == -1            # SKEL_EINVAL
    assert "device memory" in str(e.value)
