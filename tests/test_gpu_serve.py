"""The request server (cbct_server_*): continuous batching of whole reconstructions.

* every request's result is the same alone (cbct_reconstruct_ex) and in a mix of
  concurrently running requests of other shapes, view counts and storage types: the
  kernels are deterministic and requests share no device state, so the bar is equality;
* a served request matches the FP64 oracle within relative L2 1e-3;
* admission respects the slot count and the device-memory budget, and requests
  submitted while another runs are admitted and finish before it;
* failures stay with their request (non-finite input), and bad submissions are rejected
  before anything is queued.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1008_2042_gb300 import build
    build.build()
    import paper_1008_2042_gb300 as m
    m.load_library()
    return m


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def pinned(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32).pin_memory()


def case(geom, seed, photons=1e5):
    f_true = synth.voxelize(geom, synth.random_ellipsoids(geom, seed))
    return synth.noisy_line_integrals(oracle.project(geom, f_true), photons, seed + 1000)


MIX = [
    # (geometry, levels, iters, storage)
    (synth.config_small(), 1, [6], "f32"),
    (synth.config_small(24), 2, [3, 4], "bf16"),
    (synth.Geometry(nx=48, ny=40, nz=12, dx=1.2, dy=1.1, dz=1.3, nu=96, nv=28, du=0.9, dv=0.9, n_views=30),
     1, [5], "f16"),
    (synth.Geometry(nx=37, ny=29, nz=11, dx=1.7, dy=2.3, dz=1.1, nu=45, nv=23, du=1.9, dv=1.3,
                    u_off=2.1, v_off=-1.7, n_views=7, angles=tuple(0.05 + 2 * np.pi * np.arange(7) / 7)),
     3, [2, 2, 3], "f32"),
    (synth.config_small(60), 1, [4], "bf16"),
    (synth.config_small(), 3, [2, 3, 3], "f16"),
]
MU = 5e-4


@pytest.fixture(scope="module")
def mix_inputs():
    return [case(geom, 700 + i) for i, (geom, _, _, _) in enumerate(MIX)]


@pytest.fixture(scope="module")
def alone(cb, mix_inputs):
    outs = []
    for (geom, levels, iters, st), y in zip(MIX, mix_inputs):
        with cb.Geometry(geom) as g:
            yd = torch.tensor(y, dtype=torch.float32, device="cuda")
            outs.append(cb.reconstruct(g, yd, MU, levels, iters, storage=st).cpu().numpy())
    return outs


@pytest.mark.parametrize("use_graphs,priority", [(True, "size"), (False, "size"), (True, "age"), (False, "none")])
def test_results_are_the_same_alone_and_in_the_mix(cb, mix_inputs, alone, use_graphs, priority):
    """Under age priority a request's steps move between streams as it moves up the ranks;
    the result is still bit-identical to the request alone."""
    with cb.Server(max_active=4, use_graphs=use_graphs, priority=priority) as srv:
        ids, outs = [], []
        for rep in range(2):  # every request twice, so the mix holds more than the slots
            for (geom, levels, iters, st), y in zip(MIX, mix_inputs):
                out = torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory()
                ids.append(srv.submit(geom, pinned(y), MU, levels, iters, out, storage=st))
                outs.append(out)
        for rid in ids:
            srv.wait(rid, timeout=120)
        stats = srv.stats()
    assert stats["completed"] == len(ids) and stats["failed"] == 0
    assert 1 < stats["max_active_seen"] <= 4
    for i, out in enumerate(outs):
        assert np.array_equal(out.numpy(), alone[i % len(MIX)]), (i, rel(out.numpy(), alone[i % len(MIX)]))


def test_served_request_matches_the_oracle(cb):
    geom = synth.config_small()
    y = case(geom, 1001)
    out = torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory()
    with cb.Server(max_active=2) as srv:
        srv.wait(srv.submit(geom, pinned(y), MU, 1, [20], out), timeout=120)
    ref = oracle.reconstruct(geom, y, MU, 1, [20])
    assert rel(out.numpy(), ref) <= 1e-3, rel(out.numpy(), ref)


def test_admission_respects_the_memory_budget(cb, mix_inputs):
    geom, levels, iters, st = MIX[0]
    y = mix_inputs[0]
    with cb.Server(max_active=8) as probe:
        out = torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory()
        need = probe.wait(probe.submit(geom, pinned(y), MU, levels, iters, out))["device_bytes"]
    with cb.Server(budget_bytes=int(2.5 * need), max_active=8) as srv:
        ids, outs = [], []
        for _ in range(6):
            out = torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory()
            ids.append(srv.submit(geom, pinned(y), MU, levels, iters, out))
            outs.append(out)
        for rid in ids:
            srv.wait(rid, timeout=120)
        stats = srv.stats()
        # a request larger than the whole budget is refused at submission
        big = synth.config_small(400)
        with pytest.raises(cb.CbctError) as e:
            srv.submit(big, pinned(np.zeros(big.proj_shape)), MU, 1, [1],
                       torch.empty(big.vol_shape).pin_memory())
        assert e.value.status == 1
    assert stats["max_active_seen"] <= 2
    assert stats["max_bytes_seen"] <= 2.5 * need
    for out in outs:
        assert np.array_equal(out.numpy(), outs[0].numpy())


def test_requests_join_while_another_runs(cb):
    big = synth.Geometry(nx=256, ny=256, nz=64, dx=1.0, dy=1.0, dz=1.0, nu=256, nv=192, du=1.5, dv=1.5,
                         n_views=60)
    y_big = synth.random_projections(big, 9, 0.0, 3.0)
    small = synth.config_small(20)
    y_small = case(small, 1005)
    with cb.Server(max_active=4) as srv:
        out_big = torch.empty(big.vol_shape, dtype=torch.float32).pin_memory()
        rb = srv.submit(big, pinned(y_big), MU, 3, [10, 15, 20], out_big)
        smalls = []
        for _ in range(3):
            o = torch.empty(small.vol_shape, dtype=torch.float32).pin_memory()
            smalls.append(srv.submit(small, pinned(y_small), MU, 1, [3], o))
        infos = [srv.wait(r, timeout=120) for r in smalls]
        ib = srv.wait(rb, timeout=300)
    for i in infos:
        assert i["t_admit"] < ib["t_done"] and i["t_done"] < ib["t_done"]


@pytest.mark.parametrize("priority", ["size", "age"])
def test_a_failing_request_does_not_disturb_the_others(cb, mix_inputs, priority):
    geom, levels, iters, st = MIX[0]
    y = mix_inputs[0].copy()
    bad = y.copy()
    bad[0, 0, 0] = np.nan
    with cb.Server(max_active=2, priority=priority) as srv:
        o1 = torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory()
        o2 = torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory()
        r_bad = srv.submit(geom, pinned(bad), MU, levels, iters, o1)
        r_ok = srv.submit(geom, pinned(y), MU, levels, iters, o2)
        with pytest.raises(cb.CbctError) as e:
            srv.wait(r_bad, timeout=120)
        assert e.value.status == 4
        srv.wait(r_ok, timeout=120)
        stats = srv.stats()
    assert stats["failed"] == 1 and stats["completed"] == 1


def test_bad_submissions_are_rejected(cb, mix_inputs):
    geom, levels, iters, st = MIX[0]
    y = mix_inputs[0]
    with cb.Server(max_active=1) as srv:
        out = torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory()
        with pytest.raises(TypeError):  # pageable host memory
            srv.submit(geom, torch.tensor(y, dtype=torch.float32), MU, levels, iters, out)
        with pytest.raises(cb.CbctError) as e:
            srv.submit(geom, pinned(y), MU, levels, iters, out, lam=0.1)
        assert e.value.status == 5
        with pytest.raises(cb.CbctError) as e:
            srv.wait(12345)
        assert e.value.status == 1
        assert srv.stats()["submitted"] == 0


def test_l2_bound_serialises_large_volumes_and_lets_small_ones_pass(cb):
    geom = synth.config_small()           # 256 KiB volume
    tiny = synth.Geometry(nx=16, ny=16, nz=4, dx=2.0, dy=2.0, dz=2.0, nu=32, nv=8, du=3.0, dv=3.0, n_views=12)
    y = case(geom, 1001)
    y_tiny = case(tiny, 1009)
    vol = 4 * geom.nx * geom.ny * geom.nz
    with cb.Server(max_active=8, l2_budget_bytes=int(1.2 * vol)) as srv:
        outs = [torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        o_tiny = torch.empty(tiny.vol_shape, dtype=torch.float32).pin_memory()
        rx = srv.submit(geom, pinned(y), MU, 1, [20], outs[0])
        ry = srv.submit(geom, pinned(y), MU, 1, [20], outs[1])      # does not fit beside rx
        rz = srv.submit(tiny, pinned(y_tiny), MU, 1, [2], o_tiny)   # fits: overtakes ry
        ix, iy, iz = (srv.wait(r, timeout=120) for r in (rx, ry, rz))
        stats = srv.stats()
    assert iy["t_admit"] >= ix["t_done"]          # the two large volumes never overlapped
    assert iz["t_admit"] < iy["t_admit"]
    assert stats["bypassed"] >= 1
    assert np.array_equal(outs[0].numpy(), outs[1].numpy())


def test_age_priority_finishes_the_oldest_request_first(cb):
    """Under age priority the oldest admitted request's thread blocks go first: of two equal
    requests submitted back to back, the first finishes first, and both give the same
    volume as the request alone."""
    geom = synth.Geometry(nx=128, ny=128, nz=32, dx=2.0, dy=2.0, dz=2.0, nu=128, nv=48, du=3.0, dv=3.0,
                          n_views=40)
    y = synth.random_projections(geom, 11, 0.0, 2.0)
    with cb.Geometry(geom) as g:
        ref = cb.reconstruct(g, torch.tensor(y, dtype=torch.float32, device="cuda"), MU, 2, [4, 6]).cpu().numpy()
    with cb.Server(max_active=4, priority="age") as srv:
        outs = [torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory() for _ in range(3)]
        ids = [srv.submit(geom, pinned(y), MU, 2, [4, 6], o) for o in outs]
        infos = [srv.wait(r, timeout=120) for r in ids]
        stats = srv.stats()
    assert stats["completed"] == 3 and stats["max_active_seen"] >= 2
    # completions are seen by the server's polling (every 50 us): allow one poll interval
    assert infos[0]["t_done"] <= min(infos[1]["t_done"], infos[2]["t_done"]) + 1e-3
    for o in outs:
        assert np.array_equal(o.numpy(), ref)


def test_priority_option_is_checked(cb):
    with pytest.raises(ValueError):
        cb.Server(priority="fastest")
