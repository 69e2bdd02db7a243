"""Host logic of the group layer (paper_2606_31061_b300.group.plan_buckets), no GPU: one
batch per distinct shape in order of first appearance, members in input order, batches
split at the library's batch limit."""
from paper_2606_31061_b300 import group, ttals


def test_buckets_by_shape_in_order():
    specs = [((128, 128), (8, 8)), ((256, 256), (16, 16)), ((128, 128), (8, 8)), ((128, 128), (16, 16)),
             ((256, 256), (16, 16))]
    plan = group.plan_buckets(specs)
    assert [(d, r, m) for d, r, m in plan] == [
        ((128, 128), (8, 8), [0, 2]), ((256, 256), (16, 16), [1, 4]), ((128, 128), (16, 16), [3])]


def test_buckets_split_at_the_batch_limit():
    specs = [((64, 64), (4, 4))] * (2 * ttals.MAX_BATCH + 3)
    plan = group.plan_buckets(specs)
    assert [len(m) for _, _, m in plan] == [ttals.MAX_BATCH, ttals.MAX_BATCH, 3]
    assert sum((m for _, _, m in plan), []) == list(range(len(specs)))
    assert [len(m) for _, _, m in group.plan_buckets(specs[:10], max_batch=4)] == [4, 4, 2]


def test_c4_workload_has_fifteen_shapes():
    import bench
    plan = group.plan_buckets(bench.c4_specs())
    assert len(plan) == 15 and sum(len(m) for _, _, m in plan) == 64


def test_tuner_coordinate_search():
    """The tuner's search with a fake timer: environment kinds first (library defaults for the
    rest), then the solve tiles with the best kind, then the factor clusters; candidates that
    cannot run (None) are skipped; the fastest timed candidate wins."""
    from paper_2606_31061_b300 import tune
    cost = {1: 5.0, 2: 3.0, 3: 4.0, 4: None}          # environment kinds (4 does not run)
    seen = []

    def fake(sched):
        seen.append(tuple(sched[k] for k in tune.KEYS))
        c = cost[sched["env_kernel"]]
        if c is None:
            return None
        c += {(0, 0): 0.5, (2, 0): 0.2, (1, 1): 0.9, (1, 2): 0.3, (1, 4): 0.1, (1, 8): 0.4}[
            (sched["solve_kernel"], sched["k1_split"])]
        return c + {0: 0.05, 4: 0.0, 8: 0.07}[sched["factor_cluster"]]

    best = tune.coordinate_search(fake)
    assert best["env_kernel"] == 2 and best["solve_kernel"] == 1 and best["k1_split"] == 4
    assert best["factor_cluster"] == 4
    assert abs(best["ms_per_step"] - 3.1) < 1e-12
    # 4 kinds, 5 solve tiles with kind 2, 2 clusters: no candidate timed twice
    assert len(seen) == 4 + 5 + 2 and len(set(seen)) == len(seen)
    assert len(best["tried"]) == 3 + 5 + 2
    assert tune.coordinate_search(lambda sched: None) is None
