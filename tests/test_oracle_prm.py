"""Pins of the oracle's PRM exploration (Algorithm 2): node draws against the IK seed generator and
a brute-force collision test, the k nearest neighbours against a brute-force sort, the roadmap
graph against brute-force edge checks, the query's shortest path against scipy's Dijkstra on the
same graph, ResampleLinear against interpolation along the polyline, and the trajectory refinement
from given initial states against the linear-initialiser solve."""
import math

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import dijkstra

from paper_2607_11340_gb300 import synth

KEY = 0x5EED_0002
SPEC = synth.RobotSpec(L=synth.ROBOT_3SEG.L, rc=0.005, umax=0.01, nb=4)


def _rb(orc, spec=SPEC):
    return orc.make_robot(list(spec.L), spec.rc, spec.umax, thmax=spec.thmax, nb=spec.nb, rbody=spec.body_radius)


def _scene(orc, n_spheres=24, seed=7):
    rb = _rb(orc)
    us, goal, sph, ug = synth.traj_workload(SPEC, 1, n_spheres, lambda u: orc.fk(rb, u, backbone=True), seed=seed)
    return rb, us[0], ug[0], sph[0], goal[0]


def _collides(orc, rb, sph, x, delta=synth.WEIGHTS.delta):
    """Brute force: any backbone sample within r + r_body + delta of a sphere centre."""
    _, bb = orc.fk(rb, np.asarray(x)[None], backbone=True)
    bb = bb[0]
    for c in sph:
        dx, dy, dz = bb[:, 0] - c[0], bb[:, 1] - c[1], bb[:, 2] - c[2]
        reach = c[3] + rb.rbody + delta
        if np.any(dx * dx + dy * dy + dz * dz < reach * reach):
            return True
    return False


def _segment_blocked(orc, rb, sph, xa, xb, n_check):
    for c in range(1, n_check + 1):
        s = c / (n_check + 1)
        if _collides(orc, rb, sph, xa + s * (xb - xa)):
            return True
    return False


def _dist2(a, b):
    s = 0.0
    for q in range(len(a)):
        t = a[q] - b[q]
        s = s + t * t
    return s


def test_prm_nodes_are_the_seed_generator_draws(orc):
    """Without obstacles node i of roadmap r is attempt 0 of the SampleSeeds draw (problem r,
    seed i); with obstacles and 8 attempts it is the collision-redrawn seed of Algorithm 1's
    SampleSeeds (the same reading of "discarding" colliding draws)."""
    rb = _rb(orc)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    nodes, ok = orc.prm_sample(rb, synth.WEIGHTS.delta, None, KEY, 3, 40, 8)
    assert ok.all()
    np.testing.assert_array_equal(nodes, orc.seeds(rb, W, None, KEY, 3, 1, 40)[0])
    _, _, _, sph, _ = _scene(orc)
    nodes, ok = orc.prm_sample(rb, synth.WEIGHTS.delta, sph, KEY, 5, 40, 8)
    seeds = orc.seeds(rb, W, sph, KEY, 5, 1, 40)[0]
    np.testing.assert_array_equal(nodes[ok], seeds[ok])
    assert 0 < ok.sum() < 40 or ok.all()


def test_prm_nodes_valid_iff_collision_free(orc):
    rb, _, _, sph, _ = _scene(orc, n_spheres=40)
    nodes, ok = orc.prm_sample(rb, synth.WEIGHTS.delta, sph, KEY, 0, 60, 2)
    assert 0 < ok.sum() < 60, "the case should have both valid and invalid nodes"
    for x, v in zip(nodes, ok):
        assert _collides(orc, rb, sph, x) == (not v)
        assert np.all(np.abs(x) <= SPEC.umax + 1e-15)
        assert np.abs(x.reshape(-1, 3).sum(axis=1)).max() < 1e-15


def test_prm_knn_matches_brute_force(orc):
    rng = np.random.default_rng(3)
    N, d, k = 50, 9, 7
    nodes = rng.uniform(-0.01, 0.01, (N, d))
    nodes[10] = nodes[4]  # an exact tie in distance from every node
    ok = rng.uniform(size=N) > 0.2
    nbr = orc.prm_knn(nodes, ok, k)
    for i in range(N):
        if not ok[i]:
            assert np.all(nbr[i] == -1)
            continue
        cand = sorted((_dist2(nodes[i], nodes[j]), j) for j in range(N) if ok[j] and j != i)
        want = [j for _, j in cand[:k]] + [-1] * max(0, k - len(cand))
        assert list(nbr[i]) == want


def test_prm_knn_fewer_valid_nodes_than_k(orc):
    nodes = np.arange(12, dtype=float).reshape(4, 3)
    ok = np.array([True, False, True, True])
    nbr = orc.prm_knn(nodes, ok, 5)
    assert list(nbr[0]) == [2, 3, -1, -1, -1]
    assert list(nbr[1]) == [-1] * 5
    assert list(nbr[3]) == [2, 0, -1, -1, -1]


def test_prm_graph_matches_brute_force_edges(orc):
    rb, _, _, sph, _ = _scene(orc, n_spheres=24)
    N, k, nc = 40, 5, 4
    rm = orc.prm_build(rb, synth.WEIGHTS.delta, sph, KEY, 1, N, k, nc, 8)
    row, col, wt, nodes, nbr = rm["row"], rm["col"], rm["wt"], rm["nodes"], rm["nbr"]
    adj = {(i, int(col[e])): wt[e] for i in range(N) for e in range(row[i], row[i + 1])}
    listed = {(i, int(j)) for i in range(N) for j in nbr[i] if j >= 0}
    union = listed | {(j, i) for i, j in listed}
    assert set(adj) <= union
    assert all((j, i) in adj and adj[(j, i)] == w for (i, j), w in adj.items())
    blocked = 0
    for i, j in union:
        if i > j:
            continue
        free = not _segment_blocked(orc, rb, sph, nodes[i], nodes[j], nc)
        assert ((i, j) in adj) == free
        blocked += not free
        if free:
            assert adj[(i, j)] == pytest.approx(np.linalg.norm(nodes[i] - nodes[j]), rel=1e-14)
    assert blocked > 0 and len(adj) > 0
    for i in range(N):  # rows ascending
        assert np.all(np.diff(col[row[i]:row[i + 1]]) > 0)


def _query_graph(orc, rb, sph, rm, k, nc, us, ug):
    """The query graph rebuilt by brute force: the roadmap plus start / goal links."""
    nodes, ok = rm["nodes"], rm["ok"]
    N = len(nodes)
    V = N + 2
    A = np.zeros((V, V))
    for i in range(N):
        for e in range(rm["row"][i], rm["row"][i + 1]):
            A[i, rm["col"][e]] = rm["wt"][e]
    for v, q in ((N, us), (N + 1, ug)):
        cand = sorted((_dist2(q, nodes[j]), j) for j in range(N) if ok[j])[:k]
        for d2, j in cand:
            if not _segment_blocked(orc, rb, sph, q, nodes[j], nc):
                A[v, j] = A[j, v] = math.sqrt(d2)
    return A


def test_prm_query_shortest_path_and_resample(orc):
    rb, us, ug, sph, _ = _scene(orc, n_spheres=24, seed=11)
    N, k, nc, T = 60, 6, 4, 17
    rm = orc.prm_build(rb, synth.WEIGHTS.delta, sph, KEY, 0, N, k, nc, 8)
    X, length, hops, path = orc.prm_query(rb, synth.WEIGHTS.delta, sph, rm, k, nc, us, ug, T)
    A = _query_graph(orc, rb, sph, rm, k, nc, us, ug)
    dist = dijkstra(csr_matrix(A), directed=False, indices=N)
    assert np.isfinite(dist[N + 1]), "the case should have a path"
    assert length == pytest.approx(dist[N + 1], rel=1e-13)
    assert hops == len(path) - 1 >= 2 and path[0] == N and path[-1] == N + 1
    assert all(A[a, b] > 0 for a, b in zip(path[:-1], path[1:]))
    assert sum(A[a, b] for a, b in zip(path[:-1], path[1:])) == pytest.approx(length, rel=1e-13)
    # ResampleLinear: equal arc-length points of the polyline through the path's states
    P = np.array([us if v == N else ug if v == N + 1 else rm["nodes"][v] for v in path])
    cum = np.concatenate([[0.0], np.cumsum(np.linalg.norm(np.diff(P, axis=0), axis=1))])
    s = np.linspace(0.0, cum[-1], T)
    want = np.stack([np.interp(s, cum, P[:, a]) for a in range(P.shape[1])], axis=1)
    np.testing.assert_allclose(X, want, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(X[0], us)
    np.testing.assert_array_equal(X[-1], ug)


def test_prm_query_without_path_is_linear(orc):
    """A roadmap with no valid node (every draw collides): no path, the linear initialiser."""
    rb, us, ug, _, _ = _scene(orc)
    _, bb = orc.fk(rb, np.zeros((1, SPEC.d)), backbone=True)
    sph = np.array([[0.0, 0.0, 0.0, 1.0]])  # engulfs every backbone
    rm = orc.prm_build(rb, synth.WEIGHTS.delta, sph, KEY, 0, 8, 3, 2, 2)
    assert not rm["ok"].any() and len(rm["col"]) == 0
    X, length, hops, path = orc.prm_query(rb, synth.WEIGHTS.delta, sph, rm, 3, 2, us, ug, 9)
    assert hops == 0 and math.isinf(length) and len(path) == 0
    t = np.arange(9)[:, None] / 8
    np.testing.assert_allclose(X, us + t * (ug - us), rtol=0, atol=1e-18)


def test_prm_free_space_path_is_near_straight(orc):
    """No obstacles and a dense roadmap: the shortest path's length lies between the straight-line
    distance and a small multiple of it."""
    rb = _rb(orc)
    rng = np.random.default_rng(5)
    us, ug = synth.hexagon_states(rng, 2, SPEC.n, SPEC.umax)
    rm = orc.prm_build(rb, synth.WEIGHTS.delta, None, KEY, 0, 300, 10, 2, 1)
    assert rm["ok"].all()
    X, length, hops, path = orc.prm_query(rb, synth.WEIGHTS.delta, None, rm, 10, 2, us, ug, 12)
    straight = np.linalg.norm(ug - us)
    assert straight <= length <= 2.0 * straight
    steps = np.linalg.norm(np.diff(X, axis=0), axis=1)
    assert steps.max() <= length / 11 * (1 + 1e-9)


def test_traj_refine_from_linear_equals_solve_traj(orc):
    """The refinement from given initial states, started from the linear interpolation to the
    goal IK's state, reproduces the linear-initialiser solve."""
    spec = synth.RobotSpec(L=synth.ROBOT_3SEG.L, rc=0.005, umax=0.01, nb=4)
    rb = _rb(orc, spec)
    W = orc.make_weights(**synth.WEIGHTS.as_dict())
    us, goal, sph, _ = synth.traj_workload(spec, 2, 6, lambda u: orc.fk(rb, u, backbone=True), seed=4)
    cfg = orc.IkConfig(S=16, n_final=2, k_init=8, k_final=6, seed=9, p0=0)
    Tn = 6
    ref = orc.solve_traj(rb, W, sph, us, goal, Tn, cfg, 5, 1e-3, threads=1)
    X0 = np.zeros((2, Tn, spec.d))
    for q in range(2):
        cq = orc.IkConfig(S=16, n_final=2, k_init=8, k_final=6, seed=9, p0=q)
        ugq = orc.solve_ik(rb, W, sph[q], orc.IK6, goal[q:q + 1], cq, threads=1)["u"][0]
        X0[q] = us[q] + (np.arange(Tn)[:, None] / (Tn - 1)) * (ugq - us[q])
    out = orc.traj_refine(rb, W, sph, us, goal, X0, 5, 1e-3, threads=1)
    for key in ("x", "F", "goal_pos", "goal_rot", "speed", "accel", "lim_ok", "col_ok"):
        np.testing.assert_array_equal(out[key], ref[key])


def _tie_roadmap(first):
    """Two middle nodes A = (4, 3) and B = (4, -3) between start (0, 0) and goal (8, 0) (3-4-5
    triangles: every weight is exactly 5, both paths exactly 10), no roadmap edges; `first` says
    which of them has index 0."""
    d = SPEC.d
    nodes = np.zeros((2, d))
    a, b = (0, 1) if first == "A" else (1, 0)
    nodes[a, :2] = (4.0, 3.0)
    nodes[b, :2] = (4.0, -3.0)
    return dict(nodes=nodes, ok=np.ones(2, bool), row=np.zeros(3, np.int32), col=np.zeros(0, np.int32),
                wt=np.zeros(0)), a


@pytest.mark.parametrize("first", ["A", "B"])
def test_prm_query_tie_takes_the_lowest_index(orc, first):
    """Exactly tied shortest paths: the path runs through the lower-index middle node, and the
    equal-arc-length states are the exact points of that polyline."""
    rb = _rb(orc)
    rm, a = _tie_roadmap(first)
    us, ug = np.zeros(SPEC.d), np.zeros(SPEC.d)
    ug[0] = 8.0
    X, length, hops, path = orc.prm_query(rb, synth.WEIGHTS.delta, None, rm, 2, 1, us, ug, 5)
    assert length == 10.0 and hops == 2
    assert list(path) == [2, 0, 3]  # start (N), the index-0 node, goal (N + 1)
    mid = rm["nodes"][0]
    want = np.zeros((5, SPEC.d))
    want[1, :2] = mid[:2] / 2
    want[2] = mid
    want[3, :2] = (mid[:2] + ug[:2]) / 2
    want[4] = ug
    np.testing.assert_array_equal(X, want)
    assert mid[1] == (3.0 if first == "A" else -3.0)
