"""GPU Born modelling (rtm_born) against the FP64 oracle's Born operator,
which the oracle's dot test pins as the exact adjoint of the migration
numerator: several shots in one batch, snapshot intervals 1, 3 and 4, FP32
and FP16 snapshots, host buffers; a batch split does not change the data."""
import numpy as np
import pytest

import oracle
from conftest import rel_l2
from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
SEIS_TOL, HALF_TOL = 1e-4, 1e-2


@pytest.fixture(scope="module")
def ctx():
    c = rtm.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def problem():
    nx, nz, nt = 160, 80, 400
    v = inputs.layered_faulted(nz, nx, 10.0, 10.0, seed=31, water_depth=100.0)
    vm = inputs.smooth(v, 10.0, 10.0, 40.0).astype(np.float32)
    refl = ((v - inputs.smooth(v, 10.0, 10.0, 40.0)) / v).astype(np.float32)  # a sharp contrast map
    s = inputs.Survey(nx, nz, 16, 10.0, 10.0, 1e-3, nt, vm, np.array([10, 80, 151], np.int32),
                      np.array([1, 2, 1], np.int32), np.arange(0, nx, 3, dtype=np.int32),
                      np.full(len(range(0, nx, 3)), 1, np.int32), inputs.ricker(18.0, 1e-3, nt))
    return s, vm, refl


def _oracle(s, vm, refl, isnap):
    g = oracle.grid(*s.grid_tuple())
    w = s.wavelet.astype(np.float32).astype(np.float64)
    return np.stack([oracle.born(g, vm.astype(np.float64), s.src_ix[k], s.src_iz[k], s.rec_ix,
                                 s.rec_iz, w, isnap, refl.astype(np.float64))
                     for k in range(len(s.src_ix))])


def _gpu(ctx, s, vm, refl, isnap, dtype=rtm.SNAP_F32, host=False):
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    out = np.zeros((len(s.src_ix), s.nt, len(s.rec_ix)), np.float32)
    if host:
        ctx.born(rtm.make_grid(*s.grid_tuple()), vm, acq, refl, rtm.Opts(isnap, dtype, 1e-6, 0), out)
        return out
    d = torch.from_numpy(out).cuda()
    ctx.born(rtm.make_grid(*s.grid_tuple()), torch.from_numpy(vm).cuda(), acq,
             torch.from_numpy(refl).cuda(), rtm.Opts(isnap, dtype, 1e-6, 0), d)
    torch.cuda.synchronize()
    return d.cpu().numpy()


@pytest.mark.parametrize("isnap", [1, 3, 4])
def test_born_matches_oracle(ctx, problem, isnap):
    s, vm, refl = problem
    want = _oracle(s, vm, refl, isnap)
    got = _gpu(ctx, s, vm, refl, isnap)
    for k in range(len(s.src_ix)):
        assert rel_l2(got[k], want[k]) <= SEIS_TOL, (isnap, k)


def test_born_half_snapshots_and_host_buffers(ctx, problem):
    s, vm, refl = problem
    want = _oracle(s, vm, refl, 4)
    got = _gpu(ctx, s, vm, refl, 4, dtype=rtm.SNAP_F16, host=True)
    assert max(rel_l2(got[k], want[k]) for k in range(len(s.src_ix))) <= HALF_TOL


def test_born_batch_split_is_invariant(ctx, problem):
    s, vm, refl = problem
    full = _gpu(ctx, s, vm, refl, 4)
    ctx.set_batch(1)
    try:
        one = _gpu(ctx, s, vm, refl, 4)
    finally:
        ctx.set_batch(0)
    assert np.array_equal(full, one)


def test_born_refuses_checkpoint_mode(ctx, problem):
    s, vm, refl = problem
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    out = np.zeros((len(s.src_ix), s.nt, len(s.rec_ix)), np.float32)
    with pytest.raises(rtm.RTMError) as ei:
        ctx.born(rtm.make_grid(*s.grid_tuple()), vm, acq, refl, rtm.Opts(4, rtm.SNAP_F32, 1e-6, 0, 80),
                 out)
    assert ei.value.code == rtm.RTM_ERR_ARG


def test_two_step_born_matches_single_step_bitwise(ctx, problem):
    """The two-step kernel injects c m S in both substeps (its extended ring
    included) with the single-step kernel's rounding: the data agree bit for
    bit, for even and odd isnap, odd nt and half-precision snapshots."""
    import os

    s, vm, refl = problem
    s = inputs.Survey(s.nx, s.nz, s.nb, s.dx, s.dz, s.dt, 301, s.vel, s.src_ix, s.src_iz,
                      s.rec_ix, s.rec_iz, s.wavelet[:301])
    old = os.environ.get("RTM_STEP_KERNEL")
    os.environ["RTM_STEP_KERNEL"] = "1"
    try:
        one = rtm.Context(0)
    finally:
        if old is None:
            del os.environ["RTM_STEP_KERNEL"]
        else:
            os.environ["RTM_STEP_KERNEL"] = old
    try:
        for isnap, mode in ((4, rtm.SNAP_F32), (3, rtm.SNAP_F32), (1, rtm.SNAP_F32),
                            (4, rtm.SNAP_F16), (2, rtm.SNAP_BF16)):
            a = _gpu(one, s, vm, refl, isnap, dtype=mode)
            b = _gpu(ctx, s, vm, refl, isnap, dtype=mode)
            assert np.array_equal(a, b), (isnap, mode)
    finally:
        one.close()


def _adjoint(ctx, s, vm, data, isnap, dtype=rtm.SNAP_F32, checkpoint=0):
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
    ctx.migrate_adjoint(rtm.make_grid(*s.grid_tuple()), torch.from_numpy(vm).cuda(), acq,
                        torch.from_numpy(data).cuda(), rtm.Opts(isnap, dtype, 1e-6, 1, checkpoint),
                        img)
    torch.cuda.synchronize()
    return img.cpu().numpy()


def test_adjoint_matches_oracle_numerator(ctx, problem):
    # the oracle's per-shot numerators (no normalisation, no filter), summed
    s, vm, refl = problem
    data = _oracle(s, vm, refl, 4).astype(np.float32)
    g = oracle.grid(*s.grid_tuple())
    w = s.wavelet.astype(np.float32).astype(np.float64)
    _, num, _ = oracle.migrate(g, vm.astype(np.float64), s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, w,
                               data.astype(np.float64), isnap=4, return_parts=True)
    want = num.sum(axis=0)
    assert rel_l2(_adjoint(ctx, s, vm, data, 4), want) <= 1e-3
    # checkpointed recomputation gives the same numerator
    assert np.array_equal(_adjoint(ctx, s, vm, data, 4, checkpoint=40), _adjoint(ctx, s, vm, data, 4))


@pytest.mark.parametrize("isnap,dtype", [(4, rtm.SNAP_F32), (3, rtm.SNAP_F32), (4, rtm.SNAP_F16)])
def test_dot_product_born_against_adjoint(ctx, problem, isnap, dtype):
    """<born(m), d> = <m, adjoint(d)> for a random m and random data d.  Both
    sides are FP32 propagations of the same operator pair; their rounding
    errors are independent, relative ~1e-6 per field, so the two inner
    products agree to about that: the test allows 1e-4 of their size."""
    s, vm, _ = problem
    m = (inputs.normal(61, s.nz * s.nx).reshape(s.nz, s.nx) * 0.05).astype(np.float32)
    d = (inputs.normal(62, len(s.src_ix) * s.nt * len(s.rec_ix))
         .reshape(len(s.src_ix), s.nt, len(s.rec_ix)) * 1e-3).astype(np.float32)
    bm = _gpu(ctx, s, vm, m, isnap, dtype=dtype)
    ad = _adjoint(ctx, s, vm, d, isnap, dtype=dtype)
    lhs = float(np.dot(bm.ravel().astype(np.float64), d.ravel().astype(np.float64)))
    rhs = float(np.dot(m.ravel().astype(np.float64), ad.ravel().astype(np.float64)))
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), abs(rhs)), (lhs, rhs)


def test_least_squares_migration_against_fp64_cgls(ctx, problem):
    """rtm_lsrtm (CGLS over the GPU's Born operator and its adjoint) against
    the same CGLS in FP64 over the oracle's operators, on consistent data
    d = B m_true: the misfits fall monotonically, and after 3 iterations the
    reflectivity and misfits agree with the FP64 iteration."""
    s, vm, refl = problem
    g = oracle.grid(*s.grid_tuple())
    w = s.wavelet.astype(np.float32).astype(np.float64)
    v64 = vm.astype(np.float64)

    def B(m):
        return np.stack([oracle.born(g, v64, s.src_ix[k], s.src_iz[k], s.rec_ix, s.rec_iz, w, 4, m)
                         for k in range(len(s.src_ix))])

    def BT(d):
        _, num, _ = oracle.migrate(g, v64, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, w, d, isnap=4,
                                   return_parts=True)
        return num.sum(axis=0)

    d = B(refl.astype(np.float64)).astype(np.float32).astype(np.float64)
    niter = 3
    m = np.zeros_like(v64)
    r = d.copy()
    sv = BT(r)
    p = sv.copy()
    gamma = float(np.vdot(sv, sv))
    mis = [float(np.vdot(r, r))]
    for _ in range(niter):
        q = B(p)
        alpha = gamma / float(np.vdot(q, q))
        m += alpha * p
        r -= alpha * q
        mis.append(float(np.vdot(r, r)))
        sv = BT(r)
        g2 = float(np.vdot(sv, sv))
        p = sv + (g2 / gamma) * p
        gamma = g2
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    out = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
    got = ctx.lsrtm(rtm.make_grid(*s.grid_tuple()), torch.from_numpy(vm).cuda(), acq,
                    torch.from_numpy(d.astype(np.float32)).cuda(), rtm.Opts(4, rtm.SNAP_F32, 1e-6, 0),
                    niter, out)
    torch.cuda.synchronize()
    assert all(b < a for a, b in zip(got, got[1:])), got
    assert got[-1] < 0.5 * got[0]
    assert np.allclose(got, mis, rtol=1e-3), (got, mis)
    err = rel_l2(out.cpu().numpy(), m)
    assert err <= 1e-3
    print(f"CGLS misfit {got[-1] / got[0]:.3e} of the start after {niter} iterations; "
          f"misfits within {max(abs(a / b - 1) for a, b in zip(got, mis)):.1e}, m within {err:.1e}")


def test_least_squares_migration_edge_cases(ctx, problem):
    """No iterations: the reflectivity stays zero and the one misfit is the
    data's energy.  Zero data: the gradient vanishes at the start, so the
    reflectivity stays zero and every misfit is zero.  Host buffers give the
    device result bit for bit.  Checkpoint mode and a negative iteration
    count are refused."""
    s, vm, refl = problem
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    grid = rtm.make_grid(*s.grid_tuple())
    opts = rtm.Opts(4, rtm.SNAP_F32, 1e-6, 0)
    vel = torch.from_numpy(vm).cuda()
    d = (inputs.normal(5, len(s.src_ix) * s.nt * len(s.rec_ix)) * 1e-3).astype(np.float32)
    d = d.reshape(len(s.src_ix), s.nt, len(s.rec_ix))
    out = torch.full((s.nz, s.nx), 7.0, dtype=torch.float32, device="cuda")
    got = ctx.lsrtm(grid, vel, acq, torch.from_numpy(d).cuda(), opts, 0, out)
    assert len(got) == 1 and np.isclose(got[0], float(np.vdot(d.astype(np.float64), d)), rtol=1e-6)
    assert not out.any()
    got = ctx.lsrtm(grid, vel, acq, torch.zeros(d.shape, dtype=torch.float32, device="cuda"),
                    opts, 2, out)
    assert got == [0.0, 0.0, 0.0] and not out.any()
    dev_out = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
    dev_mis = ctx.lsrtm(grid, vel, acq, torch.from_numpy(d).cuda(), opts, 1, dev_out)
    host_out = np.zeros((s.nz, s.nx), np.float32)
    host_mis = ctx.lsrtm(grid, vm, acq, d, opts, 1, host_out)
    assert host_mis == dev_mis and np.array_equal(host_out, dev_out.cpu().numpy())
    for bad_opts, niter in ((rtm.Opts(4, rtm.SNAP_F32, 1e-6, 0, 8), 1), (opts, -1)):
        with pytest.raises(rtm.RTMError) as e:
            ctx.lsrtm(grid, vel, acq, torch.from_numpy(d).cuda(), bad_opts, niter, out)
        assert e.value.code == rtm.RTM_ERR_ARG
