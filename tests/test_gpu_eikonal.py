"""GPU traveltime solver (rtm_eikonal: parallel fast sweeping, FP32) against
the FP64 fast-marching oracle: the same discrete upwind solution, so the
difference is FP32 rounding only.  Each node update rounds a few times
(relative 2^-24 each) and a traveltime accumulates along a path of at most
nz + nx nodes, so |dT| <= (nz + nx) * 4 * 2^-24 * T_max bounds it; the tests
use TOL = 2e-5 of the field's largest time, which that bound allows on
these grids, and the measured differences are well below it."""
import numpy as np
import pytest

import oracle
from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(scope="module")
def ctx():
    c = rtm.Context(0)
    yield c
    c.close()


def _model(seed, nz, nx, dz, dx):
    v = inputs.layered_faulted(nz, nx, dz, dx, seed=seed)
    return v.astype(np.float32)


def _check(T, want):
    assert np.all(np.isfinite(T))
    if want.max() == 0.0:  # a grid that is only its source
        assert np.all(T == 0.0)
        return 0.0
    err = np.abs(T.astype(np.float64) - want).max() / want.max()
    assert err <= TOL, err
    return err


@pytest.mark.parametrize("shape", [(37, 53, 10.0, 15.0), (64, 31, 12.5, 12.5), (100, 20, 10.0, 12.0),
                                   (1, 40, 10.0, 10.0), (2, 2, 5.0, 7.0), (1, 1, 10.0, 10.0)])
def test_fields_match_fast_marching(ctx, shape):
    nz, nx, dz, dx = shape
    vel = np.stack([_model(s, nz, nx, dz, dx) for s in (1, 2)])
    src_iz = np.array([0, nz - 1, nz // 2], np.int32)
    src_ix = np.array([0, nx - 1, nx // 3], np.int32)
    outs = []
    for storage in ("shared", "offchip"):
        fields = torch.zeros((2, 3, nz, nx), dtype=torch.float32, device="cuda")
        iters = ctx.eikonal(torch.from_numpy(vel).cuda(), dz, dx, src_iz, src_ix, fields=fields,
                            storage=storage)
        got = fields.cpu().numpy()
        for s in range(2):
            for k in range(3):
                want = oracle.eikonal(vel[s].astype(np.float64), dz, dx, src_iz[k], src_ix[k])
                _check(got[s, k], want)
        assert all(1 <= i <= 20 for i in iters), iters
        outs.append(got)
    # both storages run the same sweeps in the same order: identical bits
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))


def test_off_chip_fields_and_host_pointers(ctx):
    # 300 x 260 nodes do not fit in shared memory: the L2-resident path
    nz, nx, dz, dx = 300, 260, 10.0, 10.0
    vel = _model(5, nz, nx, dz, dx)[None]
    rec_iz = np.zeros(nx, np.int32)
    rec_ix = np.arange(nx, dtype=np.int32)
    times = np.zeros((1, 2, nx), np.float32)
    fields = np.zeros((1, 2, nz, nx), np.float32)
    ctx.eikonal(vel, dz, dx, [0, 150], [10, 200], rec_iz, rec_ix, times=times, fields=fields)
    for k, (iz, ix) in enumerate(((0, 10), (150, 200))):
        want = oracle.eikonal(vel[0].astype(np.float64), dz, dx, iz, ix)
        _check(fields[0, k], want)
        assert np.array_equal(times[0, k], fields[0, k, 0, :])


def test_tomography_panels_full_size(ctx):
    # 34 surface sources on the 17 km x 3.5 km model at 40 m (426 x 88),
    # receivers at every surface node; 4 ensemble samples
    nz, nx, h = 88, 426, 40.0
    base = inputs.layered_faulted(nz, nx, h, h, seed=7)
    ens = inputs.ensemble(base, h, h, 4).astype(np.float32)
    src_ix = (6 + 12 * np.arange(34)).astype(np.int32)
    src_iz = np.zeros(34, np.int32)
    rec_ix = np.arange(nx, dtype=np.int32)
    rec_iz = np.zeros(nx, np.int32)
    times = torch.zeros((4, 34, nx), dtype=torch.float32, device="cuda")
    iters = ctx.eikonal(torch.from_numpy(ens).cuda(), h, h, src_iz, src_ix, rec_iz, rec_ix,
                        times=times)
    got = times.cpu().numpy()
    for s, k in ((0, 0), (1, 17), (3, 33), (2, 5)):
        want = oracle.eikonal(ens[s].astype(np.float64), h, h, 0, src_ix[k])
        _check(got[s, k], want[0])
    assert max(iters) <= 20


def test_cap_and_bad_inputs_are_reported(ctx):
    nz, nx = 40, 60
    vel = _model(9, nz, nx, 10.0, 10.0)
    fields = torch.zeros((1, 1, nz, nx), dtype=torch.float32, device="cuda")
    d = torch.from_numpy(vel).cuda()
    with pytest.raises(rtm.RTMError) as ei:
        ctx.eikonal(d, 10.0, 10.0, [nz - 1], [nx - 1], fields=fields, max_iter=1)
    assert ei.value.code == rtm.RTM_ERR_STATE
    bad = d.clone()
    bad[3, 4] = 0.0
    with pytest.raises(rtm.RTMError) as ei:
        ctx.eikonal(bad, 10.0, 10.0, [0], [0], fields=fields)
    assert ei.value.code == rtm.RTM_ERR_ARG
    with pytest.raises(rtm.RTMError) as ei:
        ctx.eikonal(d, 10.0, 10.0, [nz], [0], fields=fields)
    assert ei.value.code == rtm.RTM_ERR_ARG
    iters = ctx.eikonal(d, 10.0, 10.0, [nz - 1], [nx - 1], fields=fields)  # still usable
    _check(fields.cpu().numpy()[0, 0],
           oracle.eikonal(vel.astype(np.float64), 10.0, 10.0, nz - 1, nx - 1))
    assert iters[0] >= 2


def test_every_tile_shape_gives_the_same_bits(ctx):
    # each tile shape updates every node from neighbours in the same state as
    # the sequential sweep, so all shapes (and both storages) agree bit for bit
    import os

    nz, nx = 45, 67
    vel = _model(3, nz, nx, 10.0, 12.0)[None]
    d = torch.from_numpy(vel).cuda()
    outs = []
    old = os.environ.get("RTM_EIK_TILE")
    try:
        for shape in ("1x1", "2x2", "2x4", "4x2"):
            os.environ["RTM_EIK_TILE"] = shape
            for storage in ("shared", "offchip"):
                f = torch.zeros((1, 2, nz, nx), dtype=torch.float32, device="cuda")
                ctx.eikonal(d, 10.0, 12.0, [0, nz - 1], [5, nx // 2], fields=f, storage=storage)
                outs.append(f.cpu().numpy().view(np.uint32))
    finally:
        if old is None:
            os.environ.pop("RTM_EIK_TILE", None)
        else:
            os.environ["RTM_EIK_TILE"] = old
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    _check(outs[0].view(np.float32)[0, 0], oracle.eikonal(vel[0].astype(np.float64), 10.0, 12.0, 0, 5))
