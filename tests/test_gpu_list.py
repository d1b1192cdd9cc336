"""GPU parity of list contraction (Section 4.2, Algorithm 2) against the CPU
oracle, bit for bit: every record after contraction equals the oracle's
(the neighbours each node had when spliced out).  The tolerance is zero:
the contraction of given lists has one correct output."""
import itertools

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import load_pip, torch_cuda

pytestmark = pytest.mark.gpu

NIL = oracle.NIL


@pytest.fixture(scope="module")
def pip():
    torch_cuda()
    return load_pip()


def gpu_contract(pip, rec: np.ndarray, eps: float = 0.5, with_stats: bool = False, **opts):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(rec).view(np.int64)).cuda()
    st = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda") if with_stats else None
    pip.list_contract(t, eps=eps, stats=st, **opts)
    pip.check()
    out = t.cpu().numpy().view(np.uint64).reshape(rec.shape)
    return out, (pip.read_stats(st) if with_stats else None)


def expected(rec: np.ndarray) -> np.ndarray:
    return oracle.list_contract(rec.copy())


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_every_list_order_small_n(pip, n):
    for F in sorted({1, 2, n}):
        for order in itertools.permutations(range(n)):
            rec = workloads.lists_from_order(np.array(order, dtype=np.uint64))
            out, _ = gpu_contract(pip, rec, fresh_per_round=F)
            assert np.array_equal(out, expected(rec)), (F, order)


@pytest.mark.parametrize("n", [2, 1000, 20011])
@pytest.mark.parametrize("F", [1, 7, 3000])
def test_closed_forms_and_chains(pip, n, F):
    # a sorted list is a dependence chain: exactly one contraction per round
    for order in (np.arange(n, dtype=np.uint64), np.arange(n, dtype=np.uint64)[::-1].copy()):
        rec = workloads.lists_from_order(order)
        out, st = gpu_contract(pip, rec, fresh_per_round=F, with_stats=True)
        assert np.array_equal(out, expected(rec))
        assert st.status == 0 and st.attempts == n + st.losers
    singles = workloads.lists_from_order(np.arange(n, dtype=np.uint64), nlists=n)
    out, st = gpu_contract(pip, singles, fresh_per_round=F, with_stats=True)
    assert np.all(out == NIL) and st.losers == 0


@pytest.mark.parametrize("n,nlists,F", [(1000, 1, 1), (65537, 1, 256), (65537, 19, 4096), (300007, 3, 30000),
                                        ((1 << 20) + 3, 1, 0), ((1 << 20) + 3, 1000, 0)])
def test_random_lists(pip, n, nlists, F):
    rec = workloads.random_lists(n, rng_seed=n + nlists, nlists=nlists)
    opts = {"fresh_per_round": F} if F else {}
    out, st = gpu_contract(pip, rec, eps=0.5, with_stats=True, **opts)
    assert np.array_equal(out, expected(rec))
    assert st.status == 0 and st.attempts == n + st.losers
    p = pip.list_plan(n, 0.5, **opts)
    assert st.rounds >= p["min_rounds"] and st.max_active <= p["max_active"]
    assert p["aux_bytes"] + p["smem_bytes"] <= p["aux_bound_bytes"]


@pytest.mark.parametrize("eps", [0.1, 0.25, 0.5, 0.75])
def test_eps_sweep(pip, eps):
    n = (1 << 18) + 11
    rec = workloads.random_lists(n, rng_seed=4, nlists=7)
    out, _ = gpu_contract(pip, rec, eps=eps)
    assert np.array_equal(out, expected(rec))


def test_launch_shapes(pip):
    n = 200003
    rec = workloads.random_lists(n, rng_seed=9, nlists=2)
    ref = expected(rec)
    for opts in (dict(grid_blocks=1), dict(grid_blocks=3, block_threads=128), dict(block_threads=256),
                 dict(fresh_per_round=n), dict(prefix_c=0.01), dict(fresh_per_round=5000, grid_blocks=64)):
        out, _ = gpu_contract(pip, rec, **opts)
        assert np.array_equal(out, ref), opts


def test_invalid_lists_are_rejected_untouched_with_full_validation(pip):
    torch = torch_cuda()
    rec = workloads.random_lists(5000, rng_seed=3)
    bad = rec.copy()
    bad[17, 1] = 4999 if int(bad[17, 1]) != 4999 else 4998  # next no longer matches its prev
    oob = rec.copy()
    oob[3, 0] = 10**9
    for broken in (bad, oob):
        t = torch.from_numpy(broken.view(np.int64)).cuda()
        pip.list_contract(t, eps=0.5, flags=pip.FLAG_VALIDATE_INPUT)
        with pytest.raises(pip.PipError) as e:
            pip.check()
        assert e.value.code == pip.PIP_EINVAL
        assert np.array_equal(t.cpu().numpy().view(np.uint64), broken)
    # valid input passes the full check
    out, _ = gpu_contract(pip, rec, flags=pip.FLAG_VALIDATE_INPUT)
    assert np.array_equal(out, expected(rec))


@pytest.mark.parametrize("which", [0, 1, 2])
def test_out_of_range_pointer_is_caught_in_flight(pip, which):
    # Without the full check, the contraction itself checks every pointer's
    # range before following it, and the call reports PIP_EINVAL.  The bad
    # pointer is planted in a node whose neighbours are both larger, so no
    # splice rewrites its record before the node is worked on.
    torch = torch_cuda()
    rec = workloads.random_lists(5000, rng_seed=4)
    idx = np.arange(5000, dtype=np.uint64)
    minima = np.nonzero(((rec[:, 0] == NIL) | (rec[:, 0] > idx)) & ((rec[:, 1] == NIL) | (rec[:, 1] > idx)))[0]
    where = int(minima[[0, len(minima) // 2, -1][which]])
    rec[where, 1] = 10**12
    t = torch.from_numpy(rec.view(np.int64)).cuda()
    pip.list_contract(t, eps=0.5, fresh_per_round=64)
    with pytest.raises(pip.PipError) as e:
        pip.check()
    assert e.value.code == pip.PIP_EINVAL
    ok = workloads.random_lists(1000, rng_seed=1)
    out, _ = gpu_contract(pip, ok)
    assert np.array_equal(out, expected(ok))


def test_cycle_is_reported(pip):
    torch = torch_cuda()
    rec = workloads.lists_from_order(np.arange(64, dtype=np.uint64))
    rec[0, 0], rec[63, 1] = 63, 0  # close the list into a ring
    t = torch.from_numpy(rec.view(np.int64)).cuda()
    pip.list_contract(t, eps=0.5, fresh_per_round=8)
    with pytest.raises(pip.PipError) as e:
        pip.check()
    assert e.value.code == pip.PIP_EINTERNAL
    # the library stays usable
    ok = workloads.random_lists(1000, rng_seed=1)
    out, _ = gpu_contract(pip, ok)
    assert np.array_equal(out, expected(ok))
