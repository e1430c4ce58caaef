"""Incremental rounds on the GPU through the C ABI against the schedule oracle.

After every round the per-tile levels and the round's radii must equal the oracle's (the
decisions are fp32 and bit-exact); after the frame the image must equal the oracle image for
the frame's final level map (2e-4 with the margin exemption), and every pixel a round
rendered must be bit-equal to the full-resolution render's pixel.
"""
import numpy as np
import pytest

import oracle
from oracle import rounds as orounds
import paper_2507_04147_gb300 as a3fr
from paper_2507_04147_gb300 import synth
import gpu_helpers as gh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _setup(n=5000, w=200, h=168, stereo=True, seed=11, tile=16):
    import torch
    scene_np = synth.uniform_scene(n, 1, seed=seed)
    cams = synth.stereo_cameras(w, h, 2.0) if stereo else [synth.pinhole_camera(w, h)]
    s = a3fr.Scene.from_numpy(scene_np, tile=tile)
    for e, c in enumerate(cams):
        s.set_camera(e, c)
    out = torch.zeros((len(cams), h, w, 3), dtype=torch.float32, device="cuda")
    return scene_np, cams, s, out


def _levels(s, eyes, n_tiles):
    import torch
    return s.buffer(a3fr.BUF_LEVELS, torch.uint8).cpu().numpy().reshape(eyes, n_tiles)


@pytest.mark.parametrize("tile", [16, 32])
def test_rounds_follow_the_schedule_and_match_the_oracle(tile):
    import torch
    scene_np, cams, s, out = _setup(tile=tile)
    eyes = len(cams)
    n_tiles = oracle.tiles(200, tile) * oracle.tiles(168, tile)
    expected = [30.0, 12.0, 0.0]
    ofv = oracle.fovea((18.0, 36.0), 0.0, (4, 2, 1))
    gfv = a3fr.Fovea((18.0, 36.0), 0.0, (4, 2, 1))
    st = torch.cuda.current_stream()
    s.begin_frame(gfv, a3fr.Rounds(expected, sir=True, sir_step_px=6.0), out=out, stream=st)
    fr = [orounds.FrameRounds(cams[e], tile, ofv, expected, True, 6.0) for e in range(eyes)]
    torch.cuda.synchronize()
    assert np.array_equal(_levels(s, eyes, n_tiles), np.stack([f.level for f in fr]))
    # a prediction, two speculative rounds, a better prediction, the final prediction
    preds = {1: [[80.0, 60.0], [78.5, 60.0]], 2: [[95.0, 70.0], [93.5, 70.0]],
             3: [[100.0, 72.0], [98.5, 72.0]]}
    schedule = [1, 0, 0, 2, 0, 3]
    for ex in schedule:
        if ex:
            s.post_prediction(ex, preds[ex])
        s.render_round(out, stream=st)
        torch.cuda.synchronize()
        for e in range(eyes):
            fr[e].round(ex, preds[ex][e] if ex else (0.0, 0.0))
        assert np.array_equal(_levels(s, eyes, n_tiles), np.stack([f.level for f in fr]))
        status = s.round_status()
        np.testing.assert_array_equal(np.array(status["radius_px"], np.float32), fr[0].r)
        assert status["exit_consumed"] == fr[0].last_exit
    assert s.round_status()["complete"] == 1
    img = out.cpu().numpy()
    full = s.render_full().cpu().numpy()
    for e in range(eyes):
        rec, rect, _ = oracle.preprocess(scene_np, cams[e], tile)
        ref = oracle.render(rec, rect, cams[e], tile, level=fr[e].level)
        print(e, gh.compare_pixels(img[e].reshape(-1, 3), ref))
        live = ref.rendered.reshape(168, 200).astype(bool)
        assert np.array_equal(img[e][live], full[e][live])
        tl = np.repeat(np.repeat(full[e][0::2, 0::2], 2, axis=0), 2, axis=1)[:168, :200]
        assert np.array_equal(img[e][~live], tl[~live])


def test_rounds_without_sir_wait_for_predictions():
    import torch
    scene_np, cams, s, out = _setup(stereo=False)
    st = torch.cuda.current_stream()
    gfv = a3fr.Fovea()
    s.begin_frame(gfv, a3fr.Rounds([20.0, 0.0], sir=False), out=out, stream=st)
    s.render_round(out, stream=st)             # no prediction yet: nothing to render
    torch.cuda.synchronize()
    assert s.round_status()["rounds"] == 0 and s.round_status()["exit_consumed"] == 0
    s.post_prediction(1, [[100.0, 84.0]])
    s.render_round(out, stream=st)
    torch.cuda.synchronize()
    before = out.clone()
    lv = s.buffer(a3fr.BUF_LEVELS, torch.uint8).clone()
    s.render_round(out, stream=st)             # no new prediction, no SIR: unchanged
    torch.cuda.synchronize()
    assert torch.equal(out, before)
    assert torch.equal(s.buffer(a3fr.BUF_LEVELS, torch.uint8), lv)
    assert s.round_status()["rounds"] == 1 and not s.round_status()["complete"]
    s.post_prediction(2, [[101.0, 83.0]])
    s.render_round(out, stream=st)
    torch.cuda.synchronize()
    assert s.round_status()["complete"] == 1


def test_round_before_begin_frame_is_not_ready():
    import torch
    scene_np, cams, s, out = _setup(stereo=False)
    with pytest.raises(a3fr.A3FRError, match="NOT_READY"):
        s.render_round(out)
    s.set_gaze([[100.0, 84.0]])
    s.render_foveated()                         # a normal render does not begin a frame
    with pytest.raises(a3fr.A3FRError, match="NOT_READY"):
        s.render_round(out)


def test_native_frame_driver_modes():
    import torch
    scene_np, cams, s, out = _setup(n=20000, w=256, h=256, stereo=True)
    from paper_2507_04147_gb300 import rounds as prounds
    gfv = a3fr.Fovea()
    f = cams[0].fx
    expected = prounds.profile_expected_distances(f_px=f, samples=20000)
    preds = prounds.synthetic_predictions([[128.0, 128.0], [128.0, 128.0]], f_px=f, seed=1)
    times = np.array(prounds.TABLE2_CUM_LATENCY_MS) * 50.0      # microseconds, scaled
    st = torch.cuda.current_stream()
    res = {}
    for mode, sir in ((0, True), (0, False), (1, True), (2, True)):
        out.zero_()
        res[(mode, sir)] = a3fr.run_frame(s.handle, gfv, a3fr.Rounds(expected, sir=sir), preds, times,
                                          out, mode=mode, stream=st)
    a = res[(0, True)]
    assert a["latency_us"] > 0 and a["exits"][-1] == 6 and a["rounds"] >= 1
    assert res[(0, False)]["exits"][-1] == 6
    # without speculation every round uses a new prediction
    ex = res[(0, False)]["exits"]
    assert all(x < y for x, y in zip(ex, ex[1:]))
    assert res[(1, True)]["latency_us"] >= times[-1]         # SFR waits for the final prediction
    assert res[(2, True)]["latency_us"] > 0                  # FRR does not wait
    # the A3FR frame ends no earlier than the final prediction
    assert a["latency_us"] >= times[-1]


def test_stalled_mailbox_write_times_out_and_keeps_the_last_prediction():
    """A tracker thread descheduled in the middle of a mailbox write (Sec. 3.3, the CPU
    slow-down that SIR is for), injected on the host: the mailbox's sequence word is held
    odd while a round runs.  The round's bounded read must give up (2^16 polls), set
    A3FR_STATUS_TIMEOUT, keep the prediction it already consumed and, with SIR on, grow the
    region around it exactly as the schedule oracle's speculative round does; the GPU stays
    usable, and once the write finishes the next round consumes the posted prediction."""
    import time
    import torch
    scene_np, cams, s, out = _setup()
    eyes = len(cams)
    tile = 16
    n_tiles = oracle.tiles(200, tile) * oracle.tiles(168, tile)
    expected = [30.0, 12.0, 0.0]
    ofv = oracle.fovea((18.0, 36.0), 0.0, (4, 2, 1))
    gfv = a3fr.Fovea((18.0, 36.0), 0.0, (4, 2, 1))
    st = torch.cuda.current_stream()
    s.begin_frame(gfv, a3fr.Rounds(expected, sir=True, sir_step_px=6.0), out=out, stream=st)
    fr = [orounds.FrameRounds(cams[e], tile, ofv, expected, True, 6.0) for e in range(eyes)]
    p1 = [[80.0, 60.0], [78.5, 60.0]]
    p2 = [[95.0, 70.0], [93.5, 70.0]]
    s.post_prediction(1, p1)
    s.render_round(out, stream=st)
    torch.cuda.synchronize()
    for e in range(eyes):
        fr[e].round(1, p1[e])
    assert s.stats(reset=True)["status"] == 0
    s.stall_mailbox(True)
    try:
        s.post_prediction(2, p2)          # written, but not published while the write is open
        t0 = time.perf_counter()
        s.render_round(out, stream=st)
        torch.cuda.synchronize()
        waited = time.perf_counter() - t0
    finally:
        s.stall_mailbox(False)
    st1 = s.stats(reset=True)
    assert st1["status"] & a3fr.STATUS_TIMEOUT, st1
    assert waited < 30.0
    status = s.round_status()
    assert status["exit_consumed"] == 1
    for e in range(eyes):
        fr[e].round(0, (0.0, 0.0))        # no readable prediction: a speculative round
    assert np.array_equal(_levels(s, eyes, n_tiles), np.stack([f.level for f in fr]))
    np.testing.assert_array_equal(np.array(status["radius_px"], np.float32), fr[0].r)
    # the write has finished: the next round reads prediction 2
    s.render_round(out, stream=st)
    torch.cuda.synchronize()
    for e in range(eyes):
        fr[e].round(2, p2[e])
    assert s.stats()["status"] == 0
    assert s.round_status()["exit_consumed"] == 2
    assert np.array_equal(_levels(s, eyes, n_tiles), np.stack([f.level for f in fr]))
    print("bounded mailbox wait gave up after %.3f s" % waited)
