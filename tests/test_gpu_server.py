"""The request server: continuous batching of solves on per-slot streams with
HBM-budget admission. Each result must be the same alone and in a mix of
concurrent requests (within the solver tolerance), and the oracle's true
residual of every result must meet 1e-10."""
import numpy as np
import pytest

from helpers import ensure_library, rel_err
from paper_2201_09004_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    ensure_library()
    from paper_2201_09004_b300 import lib
    return lib


@pytest.fixture(scope="module")
def world(L):
    dims_a, dims_b = (4, 4, 4, 8), (6, 4, 4, 6)
    out = {}
    for name, d, seed in (("a", dims_a, 901), ("b", dims_b, 902)):
        U = synth.thin_links(d, seed).numpy()
        V = synth.fat_links(d, seed + 10).numpy()
        W = synth.long_links(d, seed + 20).numpy()
        lat = L.Lattice(d)
        lat.load_gauge(L.THIN, U)
        lat.load_clover(1.05)
        lat.load_gauge(L.FAT, V)
        lat.load_gauge(L.LONG, W)
        out[name] = (d, lat, U, V, W)
    return out


def requests(L, world):
    reqs = []
    for i, (name, kind, mass) in enumerate([("a", "tmc", 0.02), ("b", "hisq", 0.03), ("b", "tmc", 0.04),
                                             ("a", "hisq", 0.01), ("a", "tmc", 0.03), ("b", "hisq", 0.05)]):
        d, lat, U, V, W = world[name]
        if kind == "tmc":
            op = L.op_params(L.WILSON_TM_CLOVER, 0.05, mass, c_sw=1.05)
            rhs = [synth.z2_source(d, 950 + i).numpy(), synth.point_source(d, (1, 1, 0, 2), 1, 2).numpy()]
        else:
            op = L.op_params(L.HISQ, mass)
            rhs = [synth.z2_source(d, 960 + i, ncomp=3).numpy()]
        sp = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=L.F16)
        reqs.append((name, kind, mass, op, sp, rhs))
    return reqs


def check_residual(orc, world, name, kind, mass, b, x):
    d, lat, U, V, W = world[name]
    if kind == "tmc":
        D = orc.Wilson(d, U, 0.05, mass, clover=orc.clover(d, U, 1.05))
    else:
        D = orc.Hisq(d, V, W, mass)
    return np.linalg.norm(b - D.apply(x)) / np.linalg.norm(b)


def test_alone_equals_in_the_mix(L, orc, world):
    reqs = requests(L, world)
    alone = []
    srv = L.Server(8 << 30, 1)
    for name, kind, mass, op, sp, rhs in reqs:
        t = srv.submit(world[name][1], op, sp, rhs)
        assert srv.wait(t, 120000)
        xs, info, times, code = srv.poll(t)
        assert code == 0
        alone.append(xs)
    srv.close()
    srv = L.Server(8 << 30, 4)
    tickets = [srv.submit(world[name][1], op, sp, rhs) for name, kind, mass, op, sp, rhs in reqs]
    stats = srv.stats()
    assert stats["queued"] + stats["running"] >= 1
    mixed = []
    for t in tickets:
        assert srv.wait(t, 120000)
        xs, info, times, code = srv.poll(t)
        assert code == 0
        assert times["submitted"] <= times["admitted"] <= times["finished"]
        mixed.append(xs)
    srv.close()
    for (name, kind, mass, op, sp, rhs), xa, xm in zip(reqs, alone, mixed):
        for b, a, m in zip(rhs, xa, xm):
            assert rel_err(m, a) < 1e-8
            assert check_residual(orc, world, name, kind, mass, b, m) <= 1e-10


def test_budget_admission_and_rejection(L, world):
    name, kind, mass, op, sp, rhs = requests(L, world)[0]
    lat = world[name][1]
    # a budget below the request's own workspace is rejected at submission
    srv = L.Server(1 << 20, 2)
    with pytest.raises(L.LqError) as e:
        srv.submit(lat, op, sp, rhs)
    assert e.value.code == L.LQ_ENOMEM
    srv.close()
    # a budget that fits one request at a time serialises admissions
    probe = L.Server(1 << 40, 1)
    need = probe.request_bytes(lat, op, sp, len(rhs))
    probe.close()
    srv = L.Server(lat.device_bytes() + int(1.5 * need), 4)
    ts = [srv.submit(lat, op, sp, rhs) for _ in range(3)]
    ends = []
    for t in ts:
        assert srv.wait(t, 120000)
        _, _, times, code = srv.poll(t)
        assert code == 0
        ends.append((times["admitted"], times["finished"]))
    srv.close()
    ends.sort()
    for (a0, f0), (a1, f1) in zip(ends, ends[1:]):
        assert a1 >= f0 - 1e-3  # the next one was admitted only after the previous finished


def test_poll_unknown_ticket_and_timeout(L, world):
    srv = L.Server(1 << 30, 1)
    with pytest.raises(L.LqError):
        srv.poll(12345)
    srv.close()


def test_small_request_overtakes_a_blocked_large_one(L):
    """A request that cannot fit next to the running one does not hold back a later,
    smaller request that does fit: the small one is admitted first, the large one
    once the running request has finished; every result converges."""
    big_dims, small_dims = (16, 16, 16, 32), (4, 4, 4, 8)
    big = L.Lattice(big_dims)
    big.load_gauge(L.THIN, synth.thin_links(big_dims, 911).cuda())
    big.load_clover(1.05)
    small = L.Lattice(small_dims)
    small.load_gauge(L.THIN, synth.thin_links(small_dims, 912).cuda())
    small.load_clover(1.05)
    op = L.op_params(L.WILSON_TM_CLOVER, 0.05, 0.02, c_sw=1.05)
    slow = L.solve_params(solver=L.CGNR, tol=1e-10, prec_sloppy=L.F64)   # keeps the first request running
    fast = L.solve_params(solver=L.MIXED_CGNR, tol=1e-10, prec_sloppy=L.F16)
    site = synth.seeded_site(big_dims, 913)
    big_rhs = [synth.point_source(big_dims, site, s, c).numpy() for s in range(4) for c in range(3)]
    small_rhs = [synth.z2_source(small_dims, 914).numpy()]
    # warm caches (clover inverses, tuned kernels) so the lattices' resident bytes are final
    for lat, sp, rhs in ((big, slow, big_rhs[:1]), (big, fast, big_rhs[:1]), (small, fast, small_rhs)):
        lat.solve(op, sp, rhs)
        lat.release_workspace()
    probe = L.Server(1 << 40, 1)
    r_big = probe.request_bytes(big, op, slow, len(big_rhs))
    r_small = probe.request_bytes(small, op, fast, 1)
    probe.close()
    assert r_small < 0.25 * r_big
    budget = big.device_bytes() + small.device_bytes() + r_big + r_small + r_big // 2
    srv = L.Server(budget, 2)
    t_run = srv.submit(big, op, slow, big_rhs)
    t_large = srv.submit(big, op, slow, big_rhs)   # cannot fit while t_run runs
    t_small = srv.submit(small, op, fast, small_rhs)
    times = {}
    for name, t in (("run", t_run), ("large", t_large), ("small", t_small)):
        assert srv.wait(t, 600000)
        _, info, tm, code = srv.poll(t)
        assert code == 0, name
        times[name] = tm
    srv.close()
    assert times["small"]["admitted"] < times["large"]["admitted"]
    assert times["small"]["finished"] < times["run"]["finished"]
    assert times["large"]["admitted"] >= times["run"]["finished"] - 1e-3
