"""eig_update_query(EIG_Q_METRICS): the handle's counters over synchronous,
rejected, batched and asynchronous updates."""
import numpy as np
import pytest

import workloads
from gpu_util import dev_colmajor, dev_vec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eu():
    import paper_1706_00773_gb300 as m

    return m


def _dev(P):
    return dict(Q=dev_colmajor(P["Q"]), lam=dev_vec(P["lam"]), K=dev_colmajor(P["K"]), sigma=P["sigma"])


def test_metrics_count_every_kind_of_update(eu):
    import torch

    h = eu.eig_update_init(0, eu.EIG_MIXED)
    try:
        m0 = eu.eig_update_query(h, eu.EIG_Q_METRICS)
        assert m0["calls"] == 0 and m0["updates"] == 0 and m0["workspace_bytes"] == 0

        P = workloads.general(300, 4, seed=1, sigma="mixed")
        d = _dev(P)
        rc, rep = eu.eig_update_rank_k(h, d["Q"], d["lam"], d["K"], P["sigma"], eu.EIG_VALUES | eu.EIG_VECTORS)
        assert rc == 0
        m1 = eu.eig_update_query(h, eu.EIG_Q_METRICS)
        assert (m1["calls"], m1["updates"], m1["eigenpairs"], m1["updates_ok"]) == (1, 1, 300, 1)
        assert m1["updates_failed"] == 0 and m1["updates_pending"] == 0
        assert m1["launches"] > 0 and m1["workspace_bytes"] > 0 and m1["workspace_allocs"] == 1

        # unsorted lambda: found on the device, the update fails with EIG_EINVAL
        bad = _dev(P)
        bad["lam"] = dev_vec(P["lam"][::-1].copy())
        rc, _ = eu.eig_update_rank_k(h, bad["Q"], bad["lam"], bad["K"], P["sigma"], eu.EIG_VALUES,
                                     raise_on_error=False)
        assert rc == eu.EIG_EINVAL
        m2 = eu.eig_update_query(h, eu.EIG_Q_METRICS)
        assert (m2["calls"], m2["updates"], m2["updates_failed"]) == (2, 2, 1)

        # a batch of three, one of them unsorted
        Ps = [workloads.general(n, 3, seed=n, sigma="psd") for n in (64, 128, 200)]
        ds = [_dev(p) for p in Ps]
        ds[1]["lam"] = dev_vec(Ps[1]["lam"][::-1].copy())
        tickets = eu.eig_update_batch(h, ds)
        torch.cuda.synchronize()
        assert [eu.eig_update_query(h, eu.EIG_Q_STATUS, t) for t in tickets] == [0, eu.EIG_EINVAL, 0]
        m3 = eu.eig_update_query(h, eu.EIG_Q_METRICS)
        assert (m3["calls"], m3["updates"], m3["eigenpairs"]) == (3, 5, 300 + 300 + 64 + 128 + 200)
        assert (m3["updates_ok"], m3["updates_failed"], m3["updates_pending"]) == (3, 2, 0)

        # asynchronous: pending until its status is read
        d = _dev(P)
        rc, _ = eu.eig_update_rank_k(h, d["Q"], d["lam"], d["K"], P["sigma"], eu.EIG_VALUES | eu.EIG_ASYNC)
        assert rc == 0
        m4 = eu.eig_update_query(h, eu.EIG_Q_METRICS)
        assert m4["updates"] == 6 and m4["updates_pending"] == 1 and m4["updates_ok"] == 3
        assert eu.eig_update_query(h, eu.EIG_Q_LAST_STATUS) == 0
        m5 = eu.eig_update_query(h, eu.EIG_Q_METRICS)
        assert (m5["updates_ok"], m5["updates_pending"]) == (4, 0)
        assert m5["updates"] == m5["updates_ok"] + m5["updates_failed"] + m5["updates_pending"]
        assert np.all(np.diff([m0["launches"], m1["launches"], m3["launches"], m5["launches"]]) >= 0)
    finally:
        eu.eig_update_destroy(h)


def test_batch_tickets_are_released_and_never_reused(eu):
    """eig_update_release frees a finished ticket; its id stays invalid even
    when the slot is reused by a later batch; the counters keep its outcome."""
    import torch

    h = eu.eig_update_init(0, eu.EIG_FP64)
    try:
        Ps = [workloads.general(n, 2, seed=n, sigma="psd") for n in (50, 90, 130)]
        ds = [_dev(p) for p in Ps]
        ds[2]["lam"] = dev_vec(Ps[2]["lam"][::-1].copy())  # fails on the device
        first = eu.eig_update_batch(h, ds)
        rel = [eu.eig_update_release(h, t) for t in first]  # possibly still running
        assert all(r in (0, eu.EIG_EBUSY) for r in rel)
        torch.cuda.synchronize()
        for t, r in zip(first, rel):
            if r == eu.EIG_EBUSY:
                assert eu.eig_update_release(h, t) == 0
        for t in first:
            assert eu.eig_update_query(h, eu.EIG_Q_STATUS, t) == eu.EIG_EINVAL
            assert eu.eig_update_release(h, t) == eu.EIG_EINVAL  # twice: unknown
        m = eu.eig_update_query(h, eu.EIG_Q_METRICS)
        assert (m["updates"], m["updates_ok"], m["updates_failed"], m["updates_pending"]) == (3, 2, 1, 0)

        ds2 = [_dev(p) for p in Ps[:2]]
        second = eu.eig_update_batch(h, ds2)
        torch.cuda.synchronize()
        assert not set(second) & set(first)  # reused slots carry a new generation
        assert [eu.eig_update_query(h, eu.EIG_Q_STATUS, t) for t in second] == [0, 0]
        for t in first:
            assert eu.eig_update_query(h, eu.EIG_Q_STATUS, t) == eu.EIG_EINVAL
        rc, rep = eu.eig_update_query(h, eu.EIG_Q_REPORT, second[1])
        assert rc == 0 and rep["n"] == 90
        assert all(eu.eig_update_release(h, t) == 0 for t in second)
        m = eu.eig_update_query(h, eu.EIG_Q_METRICS)
        assert (m["updates"], m["updates_ok"], m["updates_failed"], m["updates_pending"]) == (5, 4, 1, 0)
        # releasing touches no result: the caller's buffers hold the updates
        lam_new = ds2[0]["lam"].cpu().numpy()
        assert np.all(np.diff(lam_new) >= 0) and not np.array_equal(lam_new, Ps[0]["lam"])
    finally:
        eu.eig_update_destroy(h)
