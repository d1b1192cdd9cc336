"""GPU parity of tree contraction (Section 4.2, tree contraction under the
prefix schedule) against the CPU oracle.

Every output is checked twice, in this order:
1. without any schedule: the oracle undoes the recorded rakes, latest round
   first, back to the input, and rejects a round whose rakes overlap or
   remove a parent together with its child (the paper's only condition on the
   order of contraction);
2. bit for bit against the oracle under the schedule reading taken (fresh
   block F, active-set cap kmax = 2.5 F + 2, stated here and checked against
   the plan), which fixes every round and so the records."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import load_pip, torch_cuda

pytestmark = pytest.mark.gpu

NIL = oracle.NIL
N = None


def kmax_of(F):
    return F * 5 // 2 + 2


@pytest.fixture(scope="module")
def pip():
    torch_cuda()
    return load_pip()


def gpu_contract(pip, rec: np.ndarray, eps: float = 0.5, with_stats: bool = False, **opts):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(rec).view(np.int64)).cuda()
    st = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda") if with_stats else None
    pip.tree_contract(t, eps=eps, stats=st, **opts)
    pip.check()
    out = t.cpu().numpy().view(np.uint64).reshape(rec.shape)
    return out, (pip.read_stats(st) if with_stats else None)


def expected(rec: np.ndarray, F: int) -> np.ndarray:
    out = rec.copy()
    oracle.tree_contract(out, F, kmax_of(F))
    return out


def assert_contracted(out: np.ndarray, rec: np.ndarray, F: int, ref: np.ndarray | None = None):
    """The schedule-free check first (every rake undone to the input), then
    the records against the oracle's schedule for F."""
    rc, back = oracle.tree_uncontract(out, rec)
    assert rc == 0 and np.array_equal(back, rec)
    assert np.array_equal(out, expected(rec, F) if ref is None else ref)


def plan_F(pip, n, eps, **opts):
    """The fresh block F of the schedule the call will run (the host planner
    may lower a requested F to keep the scratch bound on this device); the
    cap follows the documented kmax = 2.5 F + 2."""
    plan = pip.tree_plan(n, eps, **opts)
    assert plan["max_active"] == kmax_of(plan["fresh_per_round"]), plan
    return plan["fresh_per_round"], plan


def check(pip, rec, F, eps=0.25, **opts):
    n = rec.shape[0]
    F_run, plan = plan_F(pip, n, eps, fresh_per_round=F, **opts)
    assert F_run <= min(F, n)
    out, st = gpu_contract(pip, rec, eps=eps, with_stats=True, fresh_per_round=F, **opts)
    assert_contracted(out, rec, F_run)
    assert st.status == 0 and st.max_active <= plan["max_active"]
    return out, st


def fromlist(rows):
    return np.array([[NIL if v is None else v for v in row] for row in rows], dtype=np.uint64)


def test_hand_worked_tree_both_schedules(pip):
    seven = fromlist([[4, N, N, 0], [4, N, N, 0], [6, N, N, 0], [5, N, N, 0], [5, 0, 1, 0], [6, 4, 3, 0],
                      [N, 2, 5, 0]])
    all_at_once = fromlist([[4, 1, 5, 1], [5, 3, N, 2], [6, 5, N, 1], [N, N, N, 0], [5, 0, 1, 0], [N, 1, 3, 0],
                            [N, 2, 5, 0]])
    one_by_one = fromlist([[4, 1, 5, 1], [5, 3, 6, 2], [6, 3, N, 3], [N, N, N, 0], [5, 0, 1, 0], [6, 1, 3, 0],
                           [N, 2, 3, 0]])
    assert plan_F(pip, 7, 0.25, fresh_per_round=7)[0] == 7
    out, st = gpu_contract(pip, seven, eps=0.25, with_stats=True, fresh_per_round=7)
    # F = 7 gives kmax = 19 >= 7: all nodes active in round 1
    assert np.array_equal(out, all_at_once) and st.rounds == 3
    out, st = gpu_contract(pip, seven, eps=0.25, with_stats=True, fresh_per_round=1)
    assert np.array_equal(out, one_by_one) and st.rounds == 7


@pytest.mark.parametrize("leaves", [2, 3, 4, 5, 7, 9, 12])
def test_small_trees_every_schedule(pip, leaves):
    for seed in range(6):
        rec = workloads.random_tree(leaves, rng_seed=100 * leaves + seed, trees=1 + seed % 2, round_fill=seed)
        n = rec.shape[0]
        for F in sorted({1, 2, 3, n}):
            check(pip, rec, F)


@pytest.mark.parametrize("leaves,trees,F", [(1000, 1, 1), (65537, 1, 256), (65537, 19, 4096),
                                            (300007, 3, 30000), ((1 << 20) + 3, 1, 5000),
                                            ((1 << 20) + 3, 1000, 20000)])
def test_random_forests(pip, leaves, trees, F):
    rec = workloads.random_tree(leaves, rng_seed=leaves + trees, trees=trees, round_fill=0xABCD)
    out, st = check(pip, rec, F)
    n = rec.shape[0]
    assert st.rounds >= (n + F - 1) // F  # F_run <= F
    # one leaf left per tree
    leaf = rec[:, 1] == NIL
    assert int((leaf & (out[:, 1] == NIL)).sum()) == trees


@pytest.mark.parametrize("eps", [0.1, 0.25, 0.5, 0.75])
def test_eps_sweep_default_plans(pip, eps):
    rec = workloads.random_tree((1 << 17) + 11, rng_seed=4, trees=7)
    n = rec.shape[0]
    F, _ = plan_F(pip, n, eps)
    out, _ = gpu_contract(pip, rec, eps=eps)
    assert_contracted(out, rec, F)


def test_result_does_not_depend_on_the_launch(pip):
    rec = workloads.random_tree(100003, rng_seed=9, trees=2)
    F = 3000  # kmax = 7502 fits even one block of 512 threads (20 items per thread)
    refs = {}
    for opts in (dict(grid_blocks=1), dict(grid_blocks=3, block_threads=128), dict(block_threads=256),
                 dict(grid_blocks=64), dict(grid_blocks=300, block_threads=512)):
        F_run, _ = plan_F(pip, rec.shape[0], 0.25, fresh_per_round=F, **opts)
        if F_run not in refs:
            refs[F_run] = expected(rec, F_run)
        out, _ = gpu_contract(pip, rec, eps=0.25, fresh_per_round=F, **opts)
        assert_contracted(out, rec, F_run, refs[F_run])


@pytest.mark.parametrize("F", [1, 7, 3000])
def test_caterpillar_is_a_chain(pip, F):
    # numbered from the bottom of the spine up, each round rakes one leaf
    L = 20011
    rec = workloads.caterpillar_tree(L)
    out, st = check(pip, rec, F)
    assert st.rounds >= L - 1
    j = np.arange(L - 1, dtype=np.uint64)
    assert np.array_equal(out[:L - 1, 0], L + j) and np.array_equal(out[:L - 1, 1], j + 1)
    assert np.array_equal(out[:L - 1, 3], j + 1)


def test_degenerate_forests(pip):
    torch = torch_cuda()
    # single leaves only: nothing to rake, records untouched
    rec = np.full((4097, 4), NIL, dtype=np.uint64)
    rec[:, 3] = 5
    out, st = gpu_contract(pip, rec, eps=0.25, with_stats=True, fresh_per_round=100)
    assert np.array_equal(out, rec) and st.losers == 0
    # n = 0 and n = 1 are no-ops
    for n in (0, 1):
        t = torch.full((n, 4), -1, dtype=torch.int64, device="cuda")
        pip.tree_contract(t, eps=0.5)
        pip.check()
        assert bool((t == -1).all())
    # the smallest tree: one internal node over two leaves, both orders
    for rows in ([[2, N, N, 0], [2, N, N, 0], [N, 0, 1, 0]], [[N, 1, 2, 0], [0, N, N, 0], [0, N, N, 0]]):
        rec = fromlist(rows)
        for F in (1, 3):
            check(pip, rec, F)


def test_invalid_forests_are_rejected_untouched_with_full_validation(pip):
    torch = torch_cuda()
    rec = workloads.random_tree(3000, rng_seed=3)
    leaf = np.nonzero(rec[:, 1] == NIL)[0]
    inner = np.nonzero(rec[:, 1] != NIL)[0]
    one_child = rec.copy()
    one_child[inner[5], 2] = NIL
    no_point_back = rec.copy()
    no_point_back[leaf[7], 0] = int(inner[0]) if int(rec[leaf[7], 0]) != int(inner[0]) else int(inner[1])
    oob = rec.copy()
    oob[leaf[3], 0] = 10**9
    for broken in (one_child, no_point_back, oob):
        t = torch.from_numpy(broken.view(np.int64)).cuda()
        pip.tree_contract(t, eps=0.5, flags=pip.FLAG_VALIDATE_INPUT)
        with pytest.raises(pip.PipError) as e:
            pip.check()
        assert e.value.code == pip.PIP_EINVAL
        assert np.array_equal(t.cpu().numpy().view(np.uint64), broken)
    # valid input passes the full check
    F, _ = plan_F(pip, rec.shape[0], 0.5, fresh_per_round=500)
    out, _ = gpu_contract(pip, rec, flags=pip.FLAG_VALIDATE_INPUT, fresh_per_round=500)
    assert_contracted(out, rec, F)


@pytest.mark.parametrize("which", ["leaf_parent", "child_word", "grandparent"])
def test_bad_pointer_is_caught_in_flight(pip, which):
    # Without the full check the contraction checks every pointer it follows
    # and reports PIP_EINVAL before using a bad one.  The bad word is planted
    # where the first round reads it before any rake can rewrite it.
    torch = torch_cuda()
    rec = workloads.random_tree(4000, rng_seed=4)
    n = rec.shape[0]
    leaf = np.nonzero(rec[:, 1] == NIL)[0]
    x = int(leaf[0])  # the smallest leaf: active and raked in round 1
    p = int(rec[x, 0])
    if which == "leaf_parent":
        rec[x, 0] = 10**12
    elif which == "child_word":
        sib_slot = 2 if int(rec[p, 1]) == x else 1
        rec[p, sib_slot] = n + 5  # x's sibling pointer
    else:
        rec[p, 0] = 10**10  # x's grandparent (the smallest leaf's parent is never the root here)
        assert int(oracle.NIL) != 10**10
    t = torch.from_numpy(rec.view(np.int64)).cuda()
    pip.tree_contract(t, eps=0.1, fresh_per_round=n)
    with pytest.raises(pip.PipError) as e:
        pip.check()
    assert e.value.code == pip.PIP_EINVAL
    ok = workloads.random_tree(1000, rng_seed=1)
    F, _ = plan_F(pip, ok.shape[0], 0.5, fresh_per_round=64)
    out, _ = gpu_contract(pip, ok, fresh_per_round=64)
    assert_contracted(out, ok, F)


def test_large_forest_in_the_bench_launch(pip):
    # 2^23 leaves at the default plan for eps = 0.5, checked by the oracle's
    # schedule and by undoing every rake
    rec = workloads.random_tree(1 << 23, rng_seed=23, trees=1)
    n = rec.shape[0]
    F, _ = plan_F(pip, n, 0.5)
    out, st = gpu_contract(pip, rec, eps=0.5, with_stats=True)
    assert st.status == 0
    assert_contracted(out, rec, F)


@pytest.mark.parametrize("opts", [dict(grid_blocks=152, fresh_per_round=400000), dict(grid_blocks=38)])
def test_phase_b_cache_path(pip, opts):
    # Plans whose blocks keep the on-chip phase-B cache (eight slots of 12 or
    # 8 bytes per thread, counted in smem_bytes): with 152 blocks every marked
    # leaf's phase B is writes only; with 38 blocks threads hold more than the
    # eight cached slots, so the cached and the re-reading paths run in the
    # same rounds.
    rec = workloads.random_tree((1 << 20) + 7, rng_seed=77, trees=3)
    n = rec.shape[0]
    F, plan = plan_F(pip, n, 0.1, **opts)
    assert plan["smem_bytes"] >= plan["grid_blocks"] * plan["block_threads"] * 64, plan
    out, st = gpu_contract(pip, rec, eps=0.1, with_stats=True, **opts)
    assert st.status == 0
    assert_contracted(out, rec, F)


@pytest.mark.parametrize("cache", [12, 8, 0])
def test_each_phase_b_cache_format(pip, cache):
    # The planner caches a marked leaf's parent, sibling and grandparent (12
    # bytes a slot) where they fit the scratch bound, else only the last two
    # (8 bytes: phase B then rewrites the record from its left word on), else
    # nothing; the plan reports which in `slots`.  A plan of each format is
    # looked up by grid size and eps, and must give the oracle's records.
    rec = workloads.random_tree(1 << 17, rng_seed=5, trees=2)
    n = rec.shape[0]
    for eps in (0.1, 0.25, 0.5):
        for gb in (4, 8, 16, 38, 76, 152):
            plan = pip.tree_plan(n, eps, grid_blocks=gb)
            c = plan["slots"]
            fmt = 12 if c and c % 12 == 0 else (8 if c else 0)
            if fmt == cache:
                break
        else:
            continue
        break
    else:
        pytest.fail(f"no plan with a {cache}-byte cache slot")
    assert plan["smem_bytes"] >= plan["grid_blocks"] * plan["block_threads"] * c
    F = plan["fresh_per_round"]
    assert plan["max_active"] == kmax_of(F)
    out, st = gpu_contract(pip, rec, eps=eps, with_stats=True, grid_blocks=gb)
    assert st.status == 0
    assert_contracted(out, rec, F)
