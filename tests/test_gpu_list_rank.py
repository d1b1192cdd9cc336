"""GPU parity of list ranking (Section 4.2: list contraction, then the
reconstruction step that distributes the values back down the contraction
tree) against the CPU oracle's definition -- each node's count of nodes
before and after it in its list -- bit for bit.  The result is unique, so
the tolerance is zero whatever the schedule."""
import itertools

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import load_pip, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pip():
    torch_cuda()
    return load_pip()


def gpu_rank(pip, rec: np.ndarray, eps: float = 0.5, with_stats: bool = False, **opts):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(rec).view(np.int64)).cuda()
    st = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda") if with_stats else None
    pip.list_rank(t, eps=eps, stats=st, **opts)
    pip.check()
    out = t.cpu().numpy().view(np.uint64).reshape(rec.shape)
    return out, (pip.read_stats(st) if with_stats else None)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_every_list_order_small_n(pip, n):
    for F in sorted({1, 2, n}):
        for order in itertools.permutations(range(n)):
            for nlists in sorted({1, min(2, n)}):
                rec = workloads.lists_from_order(np.array(order, dtype=np.uint64), nlists)
                out, _ = gpu_rank(pip, rec, fresh_per_round=F)
                assert np.array_equal(out, oracle.list_rank(rec)), (F, order, nlists)


@pytest.mark.parametrize("n", [2, 1000, 20011])
@pytest.mark.parametrize("F", [1, 7, 3000])
def test_chains_and_single_nodes(pip, n, F):
    # sorted lists are the deepest contraction trees (one splice a round)
    for order in (np.arange(n, dtype=np.uint64), np.arange(n, dtype=np.uint64)[::-1].copy()):
        rec = workloads.lists_from_order(order)
        out, st = gpu_rank(pip, rec, fresh_per_round=F, with_stats=True)
        assert np.array_equal(out, oracle.list_rank(rec))
        assert st.status == 0
    singles = workloads.lists_from_order(np.arange(n, dtype=np.uint64), nlists=n)
    out, _ = gpu_rank(pip, singles, fresh_per_round=F)
    assert np.all(out == 0)


@pytest.mark.parametrize("n,nlists,F", [(100003, 1, 977), (100003, 37, 5000), ((1 << 20) + 3, 1, 0),
                                        ((1 << 20) + 3, 1000, 20000), (3 << 18, 1, 262144)])
def test_random_lists(pip, n, nlists, F):
    rec = workloads.random_lists(n, rng_seed=n + nlists, nlists=nlists)
    opts = {"fresh_per_round": F} if F else {}
    out, st = gpu_rank(pip, rec, with_stats=True, **opts)
    want = oracle.list_rank(rec)
    assert np.array_equal(out, want)
    assert st.status == 0
    # a list's length is before + after + 1 on every node of it
    assert int((out[:, 0] + out[:, 1] + 1).sum()) == int(((want[:, 0] + want[:, 1] + 1)).sum())


@pytest.mark.parametrize("eps", [0.1, 0.25, 0.5, 0.75])
def test_eps_sweep_default_plans(pip, eps):
    rec = workloads.random_lists((1 << 17) + 11, rng_seed=4, nlists=3)
    out, _ = gpu_rank(pip, rec, eps=eps)
    assert np.array_equal(out, oracle.list_rank(rec))


def test_result_does_not_depend_on_the_launch(pip):
    rec = workloads.random_lists(200003, rng_seed=9, nlists=2)
    want = oracle.list_rank(rec)
    for opts in (dict(grid_blocks=1), dict(grid_blocks=3, block_threads=128), dict(block_threads=256),
                 dict(grid_blocks=64), dict(fresh_per_round=1500, grid_blocks=30)):
        out, _ = gpu_rank(pip, rec, **opts)
        assert np.array_equal(out, want), opts


def test_bad_pointer_is_refused(pip):
    torch = torch_cuda()
    rec = workloads.random_lists(5000, rng_seed=2)
    rec[1234, 1] = 5000  # out of range
    t = torch.from_numpy(rec.view(np.int64)).cuda()
    pip.list_rank(t, eps=0.5)
    with pytest.raises(pip.PipError) as e:
        pip.check()
    assert e.value.code == pip.PIP_EINVAL
    # with the full check first, the input is left untouched
    t = torch.from_numpy(rec.view(np.int64)).cuda()
    pip.list_rank(t, eps=0.5, flags=pip.FLAG_VALIDATE_INPUT)
    with pytest.raises(pip.PipError):
        pip.check()
    assert np.array_equal(t.cpu().numpy().view(np.uint64).reshape(rec.shape), rec)
    # the library keeps working
    ok = workloads.random_lists(5000, rng_seed=3)
    out, _ = gpu_rank(pip, ok)
    assert np.array_equal(out, oracle.list_rank(ok))


def test_scratch_is_the_list_plan(pip):
    torch = torch_cuda()
    n = 1 << 20
    p = pip.list_plan(n, 0.5)
    assert p["aux_bytes"] + p["smem_bytes"] <= p["aux_bound_bytes"]
    rec = workloads.random_lists(n, rng_seed=5)
    aux = torch.empty(p["aux_bytes"], dtype=torch.uint8, device="cuda")
    t = torch.from_numpy(rec.view(np.int64)).cuda()
    pip.list_rank(t, eps=0.5, aux=aux)
    pip.check()
    assert np.array_equal(t.cpu().numpy().view(np.uint64).reshape(rec.shape), oracle.list_rank(rec))
