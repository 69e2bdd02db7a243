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
