"""C-ABI checks that need no GPU: the library builds, loads, exports every
function that include/pip.h declares, and its planner keeps the scratch bound
of the relaxed PIP model (Section 3.2; Theorem 4.2)."""
import ctypes
import math
import os
import re

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "pip.h")


@pytest.fixture(scope="module")
def pip():
    from paper_2103_01216_gb300 import _build

    _build.build()
    import paper_2103_01216_gb300 as pip

    pip.lib()
    return pip


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(pip_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pip_shuffle", "pip_shuffle_explicit_h", "pip_shuffle_ex", "pip_plan",
                     "pip_aux_bytes", "pip_check", "pip_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(pip):
    L = pip.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_and_version(pip):
    L = pip.lib()
    for code in range(8):
        assert L.pip_status_string(code)
    assert b"sm_103a" in L.pip_version()


def test_argument_errors_are_reported_before_any_launch(pip):
    L = pip.lib()
    # eps outside (0,1), n >= 2^32, bad dtype, null A: all EINVAL without touching a GPU
    assert L.pip_shuffle(ctypes.c_void_p(256), 10, 1, 0, 0.0, None) == pip.PIP_EINVAL
    assert L.pip_shuffle(ctypes.c_void_p(256), 10, 1, 0, 1.0, None) == pip.PIP_EINVAL
    assert L.pip_shuffle(ctypes.c_void_p(256), 1 << 32, 1, 0, 0.5, None) == pip.PIP_EINVAL
    assert L.pip_shuffle(ctypes.c_void_p(256), 10, 7, 0, 0.5, None) == pip.PIP_EINVAL
    assert L.pip_shuffle(None, 10, 1, 0, 0.5, None) == pip.PIP_EINVAL
    assert L.pip_shuffle(ctypes.c_void_p(260), 10, 1, 0, 0.5, None) == pip.PIP_EINVAL  # misaligned u64
    assert L.pip_shuffle_explicit_h(ctypes.c_void_p(256), 10, 1, None, 0.5, None) == pip.PIP_EINVAL
    # n <= 1 is a no-op
    assert L.pip_shuffle(None, 0, 1, 0, 0.5, None) == pip.PIP_OK
    assert L.pip_shuffle(ctypes.c_void_p(256), 1, 1, 0, 0.5, None) == pip.PIP_OK


@pytest.mark.parametrize("dtype", ["u32", "u64", "rec128"])
@pytest.mark.parametrize("eps", [0.1, 0.25, 0.5, 0.75, 0.9])
@pytest.mark.parametrize("n", [2, 3, 100, 4097, 1 << 20, 10**9, 1 << 30, (1 << 32) - 1])
def test_plan_obeys_the_aux_bound(pip, dtype, eps, n):
    p = pip.plan(n, dtype, eps)
    x = n ** (1.0 - eps)
    assert p["aux_bound_bytes"] == math.floor(pip.AUX_C * x) + 4096
    assert p["aux_bytes"] + p["smem_bytes"] <= p["aux_bound_bytes"]
    assert 1 <= p["fresh_per_round"] <= n - 1
    assert p["driver"] in (pip.DRIVER_GRID, pip.DRIVER_CTA)
    assert p["max_active"] >= p["fresh_per_round"]
    assert p["slots"] >= 2 * p["fresh_per_round"]
    assert p["min_rounds"] == -(-(n - 1) // p["fresh_per_round"])
    assert pip.aux_bytes(n, dtype, eps) == p["aux_bytes"]


def test_driver_selection(pip):
    # small prefixes run on one block with shared-memory tables, large ones on the grid
    # (no GPU here: the cluster driver needs the device's answer, so mid-size
    # prefixes fall back to the grid on CPU)
    assert pip.plan(1 << 12, "u64", 0.5)["driver"] == pip.DRIVER_CTA
    assert pip.plan(10**9, "u64", 0.75)["driver"] == pip.DRIVER_CTA
    assert pip.plan(10**9, "u64", 0.25)["driver"] == pip.DRIVER_GRID
    assert pip.plan(1 << 12, "u64", 0.5, flags=pip.FLAG_FORCE_GRID)["driver"] == pip.DRIVER_GRID
    p = pip.plan(10**9, "u64", 0.25, flags=pip.FLAG_FORCE_CTA)
    assert p["driver"] == pip.DRIVER_CTA and p["smem_bytes"] <= 227 * 1024


def test_plan_prefix_tracks_n_to_the_one_minus_eps(pip):
    # with the default prefix constant the prefix is Theta(n^(1-eps)) (bound-limited)
    for eps in (0.25, 0.5, 0.75):
        for n in (1 << 16, 1 << 22, 1 << 28):
            F = pip.plan(n, "u64", eps)["fresh_per_round"]
            x = n ** (1.0 - eps)
            assert 0.25 * x <= F <= 4.0 * x + 1


def test_plan_overrides(pip):
    p = pip.plan(1 << 20, "u64", 0.5, fresh_per_round=7, slot_factor=8, grid_blocks=3, block_threads=256,
                 flags=pip.FLAG_FORCE_GRID)
    assert p["fresh_per_round"] == 7 and p["slots"] == 8 * 7 + 32
    assert p["grid_blocks"] == 3 and p["block_threads"] == 256
    with pytest.raises(pip.PipError):
        pip.plan(1 << 20, "u64", 0.5, slot_factor=1)
    with pytest.raises(pip.PipError):
        pip.plan(1 << 20, "u64", 0.5, block_threads=100)


def test_batch_plan_host_only(pip):
    items = (pip.BatchItem * 3)()
    for j, n in enumerate([300, 1 << 16, 1 << 22]):
        items[j].A_dev = 256 * (j + 1)
        items[j].n = n
        items[j].seed = j
    plan = pip.BatchPlan()
    assert pip.lib().pip_batch_plan_make(items, 3, pip.U32, 0.5, None, ctypes.byref(plan)) == 0
    assert plan.count == 3 and plan.total_elems == 300 + (1 << 16) + (1 << 22)
    assert 1 <= plan.fmax <= 2 * 2048 + 1
    assert plan.jobs_bytes == 256 + 3 * 40
    # per-array scratch (shared memory) stays within that array's bound
    x = (1 << 22) ** 0.5
    assert plan.smem_bytes + 256 <= pip.AUX_C * x + 4096
    items[1].n = 1 << 32
    assert pip.lib().pip_batch_plan_make(items, 3, pip.U32, 0.5, None, ctypes.byref(plan)) == pip.PIP_EINVAL


def test_host_stream_tree_and_scan_argument_errors(pip):
    L = pip.lib()
    vp = ctypes.c_void_p
    one = (vp * 1)(vp(4096))
    seeds = (ctypes.c_uint64 * 1)(1)
    # nothing to do, or nothing touched: no GPU needed
    assert L.pip_shuffle_host_stream(None, None, None, 0, 10, pip.U64, 0.5, None, 0, None) == pip.PIP_OK
    assert L.pip_shuffle_host_stream(one, one, seeds, 1, 0, pip.U64, 0.5, None, 0, None) == pip.PIP_OK
    assert L.pip_shuffle_host_stream(None, one, seeds, 1, 10, pip.U64, 0.5, None, 0, None) == pip.PIP_EINVAL
    assert L.pip_shuffle_host_stream(one, one, None, 1, 10, pip.U64, 0.5, None, 0, None) == pip.PIP_EINVAL
    assert L.pip_shuffle_host_stream(one, one, seeds, 1, 10, 9, 0.5, None, 0, None) == pip.PIP_EINVAL
    assert L.pip_shuffle_host_stream(one, one, seeds, 1, 10, pip.U64, 1.0, None, 0, None) == pip.PIP_EINVAL
    nul = (vp * 1)(None)
    assert L.pip_shuffle_host_stream(nul, one, seeds, 1, 10, pip.U64, 0.5, None, 0, None) == pip.PIP_EINVAL
    # tree contraction: eps, size and alignment checks come first; n <= 1 is a no-op
    assert L.pip_tree_contract(vp(4096), 10, 0.0, None) == pip.PIP_EINVAL
    assert L.pip_tree_contract(vp(4096), 1 << 32, 0.5, None) == pip.PIP_EINVAL
    assert L.pip_tree_contract(vp(4096 + 16), 10, 0.5, None) == pip.PIP_EINVAL  # records need 32-byte alignment
    assert L.pip_tree_contract(None, 10, 0.5, None) == pip.PIP_EINVAL
    assert L.pip_tree_contract(None, 1, 0.5, None) == pip.PIP_OK
    # scan: dtype and alignment
    assert L.pip_scan(vp(4096), 10, pip.REC128, None, None) == pip.PIP_EINVAL
    assert L.pip_scan(vp(4096 + 8), 10, pip.U64, None, None) == pip.PIP_EINVAL
    assert L.pip_scan(None, 0, pip.U32, None, None) == pip.PIP_OK


@pytest.mark.parametrize("eps", [0.1, 0.25, 0.5, 0.75])
@pytest.mark.parametrize("n", [3, 1000, 1 << 20, 2 * 10**8 - 1, (1 << 32) - 3])
def test_list_and_tree_plans_obey_the_aux_bound(pip, eps, n):
    for plan in (pip.list_plan(n, eps), pip.tree_plan(n, eps)):
        F = plan["fresh_per_round"]
        assert 1 <= F <= n
        assert plan["max_active"] == F * 5 // 2 + 2
        assert plan["aux_bytes"] + plan["smem_bytes"] <= plan["aux_bound_bytes"]
        assert plan["aux_bound_bytes"] == int(128 * n ** (1 - eps)) + 4096
    tp = pip.tree_plan(n, eps)
    assert tp["elem_bytes"] == 32 and tp["driver"] == pip.DRIVER_TREE
    # the phase-B cache: 8 slots at most, 12 or 8 bytes each, counted on chip
    assert tp["slots"] in (0, 8, 16, 32, 64, 12, 24, 48, 96)
    assert tp["smem_bytes"] >= tp["grid_blocks"] * tp["block_threads"] * tp["slots"]


def test_tree_plan_takes_the_largest_cache_that_fits(pip):
    # The phase-B cache per thread is the first of 8, 4, 2, 1 three-word
    # slots, then 8, 4, 2, 1 two-word slots, that fits the scratch bound
    # beside the plan (F fixed here); so the next larger choice must not fit.
    # The on-chip lists do not depend on the cache, so the plan's own figures
    # give what every other choice would cost.
    n, eps, F = 262142, 0.25, 40000
    seen = []
    for gb in (16, 24, 38, 48, 64, 76, 100, 152):
        plan = pip.tree_plan(n, eps, grid_blocks=gb, fresh_per_round=F)
        assert plan["fresh_per_round"] == F and plan["grid_blocks"] == gb
        c, threads = plan["slots"], gb * plan["block_threads"]
        seen.append(c)
        base = plan["aux_bytes"] + plan["smem_bytes"] - threads * c  # the plan without a cache
        assert base + threads * c <= plan["aux_bound_bytes"]
        order = [96, 48, 24, 12, 64, 32, 16, 8, 0]
        for larger in order[:order.index(c)]:
            assert base + threads * larger > plan["aux_bound_bytes"], (gb, c, larger)
    assert seen == sorted(seen, key=lambda c: [96, 48, 24, 12, 64, 32, 16, 8, 0].index(c)), seen
    assert any(c % 12 == 0 and c for c in seen) and 8 in seen and 0 in seen, seen


def test_host_stream_binding_checks_its_arguments(pip):
    import torch

    a = torch.zeros(16, dtype=torch.int64)
    b = torch.zeros(8, dtype=torch.int64)
    pip.shuffle_host_stream([], [], [])  # nothing to do
    with pytest.raises(ValueError):
        pip.shuffle_host_stream([a], [a, a], [1])  # lengths differ
    with pytest.raises(ValueError):
        pip.shuffle_host_stream([a, b], [a, b], [1, 2])  # shapes differ
    with pytest.raises(ValueError):
        pip.shuffle_host_stream([a], [a.to(torch.int32)], [1])  # dtypes differ
    with pytest.raises(ValueError):
        pip.shuffle_host_stream([a[::2]], [a[::2]], [1])  # not contiguous


def test_device_entry_points_refuse_host_tensors(pip):
    # No CPU fallback: every device entry point rejects a host tensor before
    # any launch, and leaves it untouched.
    import torch

    a = torch.arange(64, dtype=torch.int64)
    lists = torch.full((8, 2), -1, dtype=torch.int64)
    trees = torch.full((7, 4), -1, dtype=torch.int64)
    calls = [
        lambda: pip.shuffle(a, seed=1),
        lambda: pip.shuffle_batch([a, a], [1, 2]),
        lambda: pip.list_contract(lists),
        lambda: pip.tree_contract(trees),
        lambda: pip.scan(a),
    ]
    for call in calls:
        with pytest.raises((ValueError, pip.PipError)):
            call()
    assert torch.equal(a, torch.arange(64, dtype=torch.int64))
    assert bool((lists == -1).all()) and bool((trees == -1).all())


def test_noalloc_refuses_host_memory_before_any_launch(pip):
    # the no-allocation entry point is reached through the raw C ABI: it
    # checks the pointer itself and leaves host memory untouched
    import torch

    a = torch.arange(64, dtype=torch.int64)
    L = pip.lib()
    assert L.pip_shuffle_noalloc(ctypes.c_void_p(a.data_ptr()), 64, pip.DTYPES["u64"], 1, 0.5, None) == pip.PIP_EINVAL
    assert L.pip_shuffle_noalloc(ctypes.c_void_p(a.data_ptr()), 64, pip.DTYPES["u64"], 1, 1.5, None) == pip.PIP_EINVAL
    assert L.pip_shuffle_noalloc(ctypes.c_void_p(a.data_ptr()), 1, pip.DTYPES["u64"], 1, 0.5, None) == pip.PIP_OK
    assert torch.equal(a, torch.arange(64, dtype=torch.int64))


def test_planner_takes_slot_factor_3_for_bound_limited_small_prefixes(pip):
    # a small, bound-limited prefix (n = 10^9, eps = 0.5): three slots per
    # fresh swap leave room for a larger prefix than four; an explicit slot
    # factor is kept as given
    p = pip.plan(10**9, "u64", 0.5)
    p4 = pip.plan(10**9, "u64", 0.5, slot_factor=4)
    assert p["slots"] == 3 * p["fresh_per_round"] + 32
    assert p4["slots"] == 4 * p4["fresh_per_round"] + 32
    assert p["fresh_per_round"] > p4["fresh_per_round"]
    assert p["aux_bytes"] + p["smem_bytes"] <= p["aux_bound_bytes"]


def test_planner_issues_reservations_early_for_small_prefixes(pip):
    # bound-limited small prefixes (the latency-bound regime) reserve and clean
    # before the commit; large prefixes after it; a caller may force it
    E = pip.FLAG_EARLY_RESERVE
    small = pip.plan(10**9, "u64", 0.5, flags=pip.FLAG_FORCE_GRID)
    assert small["fresh_per_round"] <= 131072 and small["flags"] & E
    large = pip.plan(10**9, "u64", 0.25, flags=pip.FLAG_FORCE_GRID)
    assert large["fresh_per_round"] > 131072 and not large["flags"] & E
    assert pip.plan(10**9, "u64", 0.25, flags=pip.FLAG_FORCE_GRID | E)["flags"] & E
