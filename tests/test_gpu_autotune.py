"""The autotuner picks the fastest launch shape on the caller's own reads and
leaves a working, empty graph behind (the choice never changes the graph)."""

import pytest

from gpu_util import assert_same_graph, capacity_for, oracle_export, to_device
from paper_2401_02756_gb300 import autotune, build, dbg, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    dbg.load()


def test_tune_picks_a_candidate_and_keeps_the_graph_exact():
    rs = synth.ragged_reads(2000, 200, 31, 601)
    g = dbg.Graph(rs.k, max(capacity_for(rs), (80 << 20) // 32))
    packed, offsets = to_device(rs)
    settings = [dict(insert_path=1), dict(insert_path=1, block_threads=128, tile_reads=64),
                dict(insert_path=2, apply_unroll=2), dict(insert_path=2, apply_chunk=16)]
    best, trials = autotune.tune(g, packed, offsets, reps=1, settings=settings)
    assert best in settings and len(trials) == len(settings)
    assert all(ms > 0 for _, ms in trials)
    assert g.stats() == (0, 0)  # left empty
    g.insert(packed, offsets)
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()


def test_default_candidates_cover_both_paths():
    c = autotune.candidates(31, binned=True)
    assert {x["insert_path"] for x in c} == {1, 2}
    assert {x.get("apply_mode") for x in c if x["insert_path"] == 2} == {1, 2}
    assert all(x["insert_path"] == 1 for x in autotune.candidates(32, binned=True))


def test_tune_batch_picks_a_setting_for_every_graph():
    sets = [synth.ragged_reads(600 + 300 * i, 220, 21 + 5 * (i % 3), 610 + i) for i in range(5)]
    graphs = [dbg.Graph(rs.k, capacity_for(rs) + 100_000) for rs in sets]
    items = [(g, *to_device(rs)) for g, rs in zip(graphs, sets)]
    settings = autotune.batch_candidates()[:3]
    best, trials = autotune.tune_batch(items, reps=1, settings=settings)
    assert best in settings and [t for t, _ in trials] == settings
    assert all(0 < ms < float("inf") for _, ms in trials)
    for g, rs in zip(graphs, sets):  # left holding the graphs of the last build
        assert_same_graph(g.export(), oracle_export(rs))
    dbg.build_batch(items)
    for g, rs in zip(graphs, sets):
        assert_same_graph(g.export(), oracle_export(rs))
        g.close()
