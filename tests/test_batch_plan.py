"""Chunk planning of multi-camera workloads (host logic, no GPU)."""
import pytest

from paper_1909_04573_gb300 import batch, synth


def _check(cams, budget, chunks):
    seen = {i: [] for i in range(len(cams))}
    for ch in chunks:
        assert ch, "empty chunk"
        end = 0
        for p in ch:
            fb, m, d = cams[p.cam]
            assert p.offset % batch.ALIGN == 0 and p.offset >= end
            end = p.offset + (p.f1 - p.f0) * fb
            assert end <= budget
            assert p.f0 % d == 0 and (p.f1 % d == 0 or p.f1 == m)     # whole groups only
            seen[p.cam].extend(range(p.f0, p.f1))
    for i, (fb, m, d) in enumerate(cams):
        assert seen[i] == list(range(m))                              # every frame once, in order


@pytest.mark.parametrize("budget", [1024, 1537, 4096, 10 ** 6])
def test_plan_covers_every_frame_once(budget):
    cams = [(10, 37, 5), (100, 9, 9), (7, 101, 10), (256, 3, 1), (33, 20, 4)]
    _check(cams, budget, batch.plan_chunks(cams, budget))


def test_plan_packs_until_full():
    cams = [(256, 10, 2), (256, 10, 2)]
    chunks = batch.plan_chunks(cams, 256 * 8)
    assert [sum(p.f1 - p.f0 for p in ch) for ch in chunks] == [8, 8, 4]


def test_ragged_last_group_fills_remaining_room():
    chunks = batch.plan_chunks([(256, 7, 4)], 256 * 4)
    assert [(p.f0, p.f1) for ch in chunks for p in ch] == [(0, 4), (4, 7)]


def test_group_larger_than_budget_is_rejected():
    with pytest.raises(ValueError):
        batch.plan_chunks([(100, 50, 20)], 1000)
    with pytest.raises(ValueError):
        batch.plan_chunks([(100, 5, 6)], 10 ** 6)                      # d > m


def test_batch_workload_plan():
    specs = synth.batch_cameras()
    cams = [(c.H * c.W * c.C, m, d) for c, m, d in specs]
    assert len(specs) == 32
    assert {(c.H, c.W) for c, _, _ in specs} <= set(synth.BATCH_RESOLUTIONS)
    assert all(100 <= m <= 2000 and 10 <= d <= 100 for _, m, d in specs)
    budget = 96 << 30
    chunks = batch.plan_chunks(cams, budget)
    _check(cams, budget, chunks)
    assert len(chunks) == -(-sum(fb * m for fb, m, _ in cams) // budget)  # no chunk left half empty
