"""Host logic of the launch-shape autotuner (no GPU): the proportional subset that large
batches are tuned on."""
import paper_1209_5235_gb300.autotune as at
import paper_1209_5235_gb300.binding as b
import synth


def _items():
    src = synth.scenes.barrel_source()
    return b.make_items([(0, 10_000_000, 0, src, 0), (1, 3, 10_000_000, src, 40), (2, 0, 10_000_003, src, 80)])


def test_subset_scales_track_counts_and_keeps_the_rest():
    items = _items()
    sub = at.subset_items(items, 2_000_000)
    assert [w.n_tracks for w in sub] == [2_000_000 - 1, 1, 0]   # floor of the share, at least one, empty stays empty
    for w, v in zip(items, sub):
        assert (v.geom, v.track_id0, v.tally_offset) == (w.geom, w.track_id0, w.tally_offset)
        assert (v.source.e_kind, v.source.e0, v.source.e1, v.source.spot_sigma) == \
            (w.source.e_kind, w.source.e0, w.source.e1, w.source.spot_sigma)
        assert list(v.source.pos) == list(w.source.pos) and list(v.source.dir) == list(w.source.dir)
    assert [w.n_tracks for w in items] == [10_000_000, 3, 0]    # the caller's batch is not modified


def test_small_batches_are_tuned_whole():
    items = _items()
    assert at.subset_items(items, 0) is items
    assert at.subset_items(items, 20_000_000) is items


def test_tuner_shapes_are_valid_batch_descriptions():
    """Every shape the tuner tries (the persistent defaults and the staged shapes) fills the batch description's
    schedule fields within their ABI ranges."""
    items = _items()
    for shape in [at.DEFAULT] + [dict(at.DEFAULT, schedule=b.G4N_SCHEDULE_STAGED, **s) for s in at.STAGED]:
        d = b._desc(items, 1, 0.01, 0, 100, 200, 0, shape["block_size"], shape["blocks_per_sm"], shape["refill_min"],
                    shape["interact_min"], False, shape["walk_budget"], shape["regroup_period"], shape["schedule"],
                    shape["pool_tracks"], shape["drain_tracks"], shape["staged_flags"])
        assert d.schedule in (b.G4N_SCHEDULE_PERSISTENT, b.G4N_SCHEDULE_STAGED)
        assert d.staged_flags in (0, b.G4N_STAGED_RELOCATION_KERNEL)
        assert d.pool_tracks >= 0 and d.drain_tracks >= -1 and 0 <= d.blocks_per_sm <= 16
        assert d.block_size % 32 == 0 and d.block_size <= 128
    assert {s["drain_tracks"] for s in at.STAGED} >= {0, -1}     # the default drain point and no drain are both tried
