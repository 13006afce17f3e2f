"""The end-to-end entry point (host buffers in and out) on a batch large
enough to be cut into pipeline segments: copies of one segment overlap the
reconstruction of another. Every tile must still equal the oracle's result
(hashes stored in tests/golden/batch_hashes.json, written from the oracle
only), and a marker violation in a later segment must be reported with its
index in the whole batch."""
import hashlib
import json
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1311_0378_gb300 as rc  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "batch_hashes.json")


def _host_pairs(specs, seed):
    Is = [torch.empty((s.H, s.W), dtype=torch.uint8).pin_memory() for s in specs]
    Js = [torch.empty((s.H, s.W), dtype=torch.uint8).pin_memory() for s in specs]
    synth.generate_into(specs, seed, [x.data_ptr() for x in Is], [x.data_ptr() for x in Js])
    return Is, Js


def test_host_batch_in_segments_matches_oracle():
    import paper_1311_0378_gb300.build as b
    b.build()
    with open(GOLDEN) as f:
        gold = json.load(f)["workloads"]["batch64"]
    w = synth.workload("batch64")
    specs = list(w.tiles[:20])          # 20 x 4096^2 = 335 Mpx: four segments
    Is, Js = _host_pairs(specs, w.seed)
    digits = len(gold["tiles"][0]["R"])
    ctx = rc.recon_init(0, 0, 0)
    try:
        for rep in range(2):            # twice: the second call reuses the pipeline state
            if rep:
                Is, Js = _host_pairs(specs, w.seed)
            tiles = [(I.data_ptr(), J.data_ptr(), s.H, s.W, s.W, s.conn) for I, J, s in zip(Is, Js, specs)]
            rc.check(rc.recon_batch_host(ctx, tiles), "recon_batch_host")
            bad = [t for t, J in enumerate(Js)
                   if hashlib.sha256(memoryview(J.numpy()).cast("B")).hexdigest()[:digits] != gold["tiles"][t]["R"]]
            assert not bad, "tiles differing from the oracle: %s" % bad
    finally:
        rc.recon_free(ctx)


def test_host_batch_reports_failing_tile_of_a_later_segment():
    w = synth.workload("batch64")
    specs = list(w.tiles[:20])
    Is, Js = _host_pairs(specs, w.seed)
    Is[17][100, 200] = 200   # J > I at one pixel of tile 17 (fourth segment)
    Js[17][100, 200] = 201
    ctx = rc.recon_init(0, 0, 0)
    try:
        tiles = [(I.data_ptr(), J.data_ptr(), s.H, s.W, s.W, s.conn) for I, J, s in zip(Is, Js, specs)]
        assert rc.recon_batch_host(ctx, tiles) == rc.RECON_EMARKER
        assert rc.recon_last_error_tile(ctx) == 17
    finally:
        rc.recon_free(ctx)


def test_host_batch_learned_schedule_matches_oracle():
    """With the learned schedule, each segment is planned on a side stream
    while the segment before it runs; the results must not change."""
    from paper_1311_0378_gb300 import cost_model
    with open(GOLDEN) as f:
        gold = json.load(f)["workloads"]["batch64"]
    w = synth.workload("batch64")
    specs = list(w.tiles[:20])
    Is, Js = _host_pairs(specs, w.seed)
    digits = len(gold["tiles"][0]["R"])
    ctx = rc.recon_init(0, 0, rc.RECON_FLAG_LEARNED)
    try:
        cost_model.install(ctx)
        tiles = [(I.data_ptr(), J.data_ptr(), s.H, s.W, s.W, s.conn) for I, J, s in zip(Is, Js, specs)]
        rc.check(rc.recon_batch_host(ctx, tiles), "recon_batch_host")
        bad = [t for t, J in enumerate(Js)
               if hashlib.sha256(memoryview(J.numpy()).cast("B")).hexdigest()[:digits] != gold["tiles"][t]["R"]]
        assert not bad, "tiles differing from the oracle: %s" % bad
    finally:
        rc.recon_free(ctx)


def test_host_batch_failing_first_segment_then_normal_call():
    """A violation in the first segment is reported while the later segments
    were already queued behind it; the same context then runs a clean batch."""
    with open(GOLDEN) as f:
        gold = json.load(f)["workloads"]["batch64"]
    w = synth.workload("batch64")
    specs = list(w.tiles[:20])
    Is, Js = _host_pairs(specs, w.seed)
    Is[2][7, 9] = 50     # J > I at one pixel of tile 2 (first segment)
    Js[2][7, 9] = 60
    digits = len(gold["tiles"][0]["R"])
    ctx = rc.recon_init(0, 0, 0)
    try:
        tiles = [(I.data_ptr(), J.data_ptr(), s.H, s.W, s.W, s.conn) for I, J, s in zip(Is, Js, specs)]
        assert rc.recon_batch_host(ctx, tiles) == rc.RECON_EMARKER
        assert rc.recon_last_error_tile(ctx) == 2
        assert rc.recon_sync(ctx) == rc.RECON_EMARKER
        Is, Js = _host_pairs(specs, w.seed)
        tiles = [(I.data_ptr(), J.data_ptr(), s.H, s.W, s.W, s.conn) for I, J, s in zip(Is, Js, specs)]
        rc.check(rc.recon_batch_host(ctx, tiles), "recon_batch_host after a failure")
        assert rc.recon_last_error_tile(ctx) == -1
        bad = [t for t, J in enumerate(Js)
               if hashlib.sha256(memoryview(J.numpy()).cast("B")).hexdigest()[:digits] != gold["tiles"][t]["R"]]
        assert not bad, "tiles differing from the oracle: %s" % bad
    finally:
        rc.recon_free(ctx)
