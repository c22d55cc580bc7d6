"""GPU: uneven batches -- per-frame quantiser/LLR and the one-launch plan decoder.

* Per-frame quantiser and slice LLRs: identical, sample by sample, to the
  single-range entry points called on each frame with its own parameters, and
  against the FP64 oracle (quantiser bit-exact, LLRs within TOL).
* Plan decoder (layered offset min-sum, FP32): bits, iteration counts and
  convergence flags identical to qkdrec_decode_batch with the same options on
  every group, for every tuning the autotuner may pick; against the oracle
  directly after fixed iterations (bits where the oracle's posterior is not
  near zero, iteration counts and flags exactly); CUDA-graph capture and
  replay with the inputs refilled in place; ragged and empty groups.
"""
import numpy as np
import pytest

import oracle
import synth
from _workloads import TOL, bpsk_frames, code, rel_ok

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_08418_b300 as q  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2108_08418_b300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


# ----------------------------------------------------- per-frame quantiser / LLR
def frames_case(seed, lengths, m=5):
    lengths = np.asarray(lengths, dtype=np.int64)
    snr = synth.philox(seed).uniform(2.0, 15.0, size=lengths.size)
    x, y = synth.gaussian_frames(seed, lengths, snr)
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    rng = np.array([oracle.quantiser_range(s) for s in snr], dtype=np.float64).reshape(-1, 2)
    par = np.concatenate([rng, (snr ** -0.5)[:, None]], axis=1)
    return x, y, off, rng, par, snr


@pytest.mark.parametrize("label", ["gray", "binary"])
def test_frames_quantiser_and_llr_equal_per_frame_calls(label):
    m = 5
    lengths = [1000, 0, 1, 4097, 333, 2048]
    x, y, off, rng, par, snr = frames_case(700, lengths, m)
    idx, bits = q.qkdrec_quantise_slices_frames(dev(y), dev(off), dev(rng), m, label)
    idx, bits = host(idx), host(bits)
    for f in range(len(lengths)):
        a, b = off[f], off[f + 1]
        if a == b:
            continue
        i1, b1 = q.qkdrec_quantise_slices(dev(y[a:b]), m, rng[f, 0], rng[f, 1], label)
        assert np.array_equal(idx[a:b], host(i1))
        assert np.array_equal(bits[:, a:b], host(b1))
        ri, rb = oracle.quantise(y[a:b], m, rng[f, 0], rng[f, 1], label)
        assert np.array_equal(idx[a:b], ri) and np.array_equal(bits[:, a:b], rb)
    for j in range(m):
        llr = host(q.qkdrec_slice_llr_frames(dev(x), dev(off), dev(par), m, j,
                                             dev(np.ascontiguousarray(bits[:j])) if j else None, label))
        for f in range(len(lengths)):
            a, b = off[f], off[f + 1]
            if a == b:
                continue
            lb = dev(np.ascontiguousarray(bits[:j, a:b])) if j else None
            one = host(q.qkdrec_slice_llr(dev(x[a:b]), m, j, rng[f, 0], rng[f, 1], par[f, 2], lb, label))
            assert np.array_equal(llr[a:b].view(np.uint32), one.view(np.uint32)), (j, f)
            if f % 2 == 0:
                ref = oracle.slice_llr(x[a:b].astype(np.float64), bits[:j, a:b], j, m, rng[f, 0], rng[f, 1],
                                       par[f, 2], label)
                assert rel_ok(llr[a:b], ref).all(), (j, f)


def test_frames_empty_batch_is_a_no_op():
    off = dev(np.zeros(1, np.int64))
    idx, bits = q.qkdrec_quantise_slices_frames(torch.zeros(0, device="cuda"), off,
                                                dev(np.zeros((0, 2))), 4)
    assert idx.numel() == 0 and bits.numel() == 0


# ------------------------------------------------------------------ plan decoder
TUNINGS = [None,
           dict(frames_per_tile=8, threads_per_cta=256, stage_depth=4, ctas_per_tile=1),
           dict(frames_per_tile=16, threads_per_cta=512, stage_depth=4, ctas_per_tile=2),
           dict(frames_per_tile=32, threads_per_cta=1024, stage_depth=4, ctas_per_tile=8),
           dict(frames_per_tile=32, threads_per_cta=256, stage_depth=16, ctas_per_tile=1),
           dict(frames_per_tile=8, threads_per_cta=512, stage_depth=8, ctas_per_tile=4),
           # several tiles of a group decoded together, layer by layer (ragged last item)
           dict(frames_per_tile=8, threads_per_cta=256, stage_depth=4, ctas_per_tile=2, tiles_per_item=2),
           dict(frames_per_tile=8, threads_per_cta=1024, stage_depth=4, ctas_per_tile=8, tiles_per_item=4),
           dict(frames_per_tile=32, threads_per_cta=512, stage_depth=8, ctas_per_tile=1, tiles_per_item=4),
           # two or four frames per lane (2- and 4-wide accesses; frames retiring inside a lane)
           dict(frames_per_tile=16, threads_per_cta=256, stage_depth=8, ctas_per_tile=2, frames_per_lane=2),
           dict(frames_per_tile=32, threads_per_cta=512, stage_depth=4, ctas_per_tile=1, frames_per_lane=4),
           dict(frames_per_tile=32, threads_per_cta=256, stage_depth=8, ctas_per_tile=8, frames_per_lane=4,
                tiles_per_item=2),
           dict(frames_per_tile=32, threads_per_cta=512, stage_depth=4, ctas_per_tile=4, frames_per_lane=2),
           # sparse mode (one (check, frame) pair per lane) never, from the first iteration, or late
           dict(frames_per_tile=8, threads_per_cta=256, stage_depth=4, ctas_per_tile=1, sparse_frames=0),
           dict(frames_per_tile=32, threads_per_cta=512, stage_depth=4, ctas_per_tile=2, frames_per_lane=4,
                tiles_per_item=4, sparse_frames=0),
           dict(frames_per_tile=32, threads_per_cta=256, stage_depth=8, ctas_per_tile=4, frames_per_lane=4,
                tiles_per_item=2, sparse_frames=8),
           dict(frames_per_tile=16, threads_per_cta=1024, stage_depth=4, ctas_per_tile=8, tiles_per_item=4,
                sparse_frames=16),
           dict(frames_per_tile=32, threads_per_cta=512, stage_depth=4, ctas_per_tile=8, frames_per_lane=4,
                tiles_per_item=2, sparse_frames=4)]


def make_groups(spec, seed=800):
    """spec: list of (n, rate, frames, sigma)."""
    out = []
    for i, (n, rate, F, sigma) in enumerate(spec):
        rp, ci, M = code(seed + 10 * i, n, rate)
        c = q.Code(n, rp, ci)
        b, llr = bpsk_frames(seed + 10 * i + 1, F, n, sigma)
        s = oracle.syndrome(rp, ci, b) if F else np.zeros((0, M), np.uint8)
        out.append(dict(code=c, rp=rp, ci=ci, b=b, llr_h=llr, synd_h=s,
                        llr=dev(llr), synd=dev(s),
                        bits=torch.empty((F, n), dtype=torch.uint8, device="cuda"),
                        iters=torch.empty(F, dtype=torch.int32, device="cuda"),
                        conv=torch.empty(F, dtype=torch.uint8, device="cuda")))
    return out


# ragged tiles, an empty group, two check-degree classes, and check degree 48 (above the
# shared-memory stash of 32 edges)
SPEC = [(1024, 0.5, 37, 0.82), (2048, 0.75, 5, 0.55), (720, 40 / 90, 70, 0.9), (512, 0.5, 0, 0.8),
        (4096, 0.5, 33, 0.86), (4096, 60 / 64, 11, 0.35)]


def reference(g, opts):
    return q.qkdrec_decode_batch(g["code"], g["llr"], g["synd"], opts)


@pytest.mark.parametrize("tuning", TUNINGS)
@pytest.mark.parametrize("early_stop,max_iter", [(True, 40), (False, 7), (False, 0), (True, 0)])
def test_plan_identical_to_batch_decoder(tuning, early_stop, max_iter):
    groups = make_groups(SPEC)
    opts = q.DecodeOpts(algo="oms_layered", prec="f32", max_iter=max_iter, early_stop=early_stop)
    plan = q.Plan(groups, opts, tuning)
    if tuning is not None:
        assert {k: plan.tuning()[k] for k in tuning} == tuning
    ws = plan.workspace()
    plan.launch(ws)
    torch.cuda.synchronize()
    for g in groups:
        if g["llr_h"].shape[0] == 0:
            continue
        ref = reference(g, opts)
        assert torch.equal(g["bits"], ref["bits"])
        assert torch.equal(g["iters"], ref["iters"])
        assert torch.equal(g["conv"], ref["converged"])
    plan.destroy()


@pytest.mark.parametrize("iters", [1, 3])
def test_plan_vs_oracle_after_fixed_iterations(iters):
    groups = make_groups([(1024, 0.5, 13, 0.85), (720, 40 / 90, 9, 0.9)], seed=850)
    opts = q.DecodeOpts(algo="oms_layered", prec="f32", max_iter=iters, early_stop=False)
    plan = q.Plan(groups, opts, dict(frames_per_tile=8, threads_per_cta=256, stage_depth=4, ctas_per_tile=4))
    plan.launch(plan.workspace())
    torch.cuda.synchronize()
    for g in groups:
        ref = oracle.decode(g["rp"], g["ci"], g["llr_h"].astype(np.float64), g["synd_h"], "oms_layered",
                            max_iter=iters, early_stop=False, offset=0.5)
        sure = np.abs(ref["post"]) > 1e-3
        assert np.array_equal(host(g["bits"])[sure], ref["bits"][sure])
        assert np.array_equal(host(g["iters"]), ref["iters"])
        assert np.array_equal(host(g["conv"]), ref["converged"])


def test_plan_full_decode_converged_words_satisfy_syndrome():
    groups = make_groups([(2048, 0.5, 64, 0.8), (4096, 0.75, 40, 0.5)], seed=870)
    opts = q.DecodeOpts(algo="oms_layered", prec="f32", max_iter=50, early_stop=True)
    plan = q.Plan(groups, opts)
    plan.launch(plan.workspace())
    torch.cuda.synchronize()
    for g in groups:
        bits, conv = host(g["bits"]), host(g["conv"])
        assert conv.mean() > 0.5
        for f in np.flatnonzero(conv):
            assert np.array_equal(oracle.syndrome(g["rp"], g["ci"], bits[f:f + 1])[0], g["synd_h"][f])
        # frames the oracle decodes to the transmitted word: the plan agrees where both converge
        ref = oracle.decode(g["rp"], g["ci"], g["llr_h"].astype(np.float64), g["synd_h"], "oms_layered",
                            max_iter=50, early_stop=True, offset=0.5)
        both = (conv == 1) & (ref["converged"] == 1)
        assert np.array_equal(bits[both], ref["bits"][both])


def test_plan_graph_capture_and_replay_with_refilled_inputs():
    groups = make_groups([(1024, 0.5, 40, 0.84), (2048, 0.75, 20, 0.55)], seed=900)
    opts = q.DecodeOpts(algo="oms_layered", prec="f32", max_iter=30, early_stop=True)
    plan = q.Plan(groups, opts)
    ws = plan.workspace()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.launch(ws, side)          # warm-up outside capture (sets kernel attributes once)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.launch(ws, torch.cuda.current_stream())
    for rep in range(2):
        for i, g in enumerate(groups):
            n, F = g["code"].n, g["llr_h"].shape[0]
            b, llr = bpsk_frames(950 + 7 * rep + i, F, n, 0.84 if i == 0 else 0.55)
            s = oracle.syndrome(g["rp"], g["ci"], b)
            g["llr"].copy_(dev(llr))
            g["synd"].copy_(dev(s))
            g["bits"].fill_(7)
        graph.replay()
        torch.cuda.synchronize()
        for g in groups:
            ref = reference(g, opts)
            assert torch.equal(g["bits"], ref["bits"])
            assert torch.equal(g["iters"], ref["iters"])
            assert torch.equal(g["conv"], ref["converged"])


def test_plan_autotune_picks_a_supported_tuning_and_keeps_results():
    groups = make_groups([(2048, 0.5, 70, 0.82), (1024, 0.75, 30, 0.55)], seed=960)
    opts = q.DecodeOpts(algo="oms_layered", prec="f32", max_iter=20, early_stop=True)
    plan = q.Plan(groups, opts)
    ws = plan.workspace()
    best, ms = plan.autotune(ws, max_iter=5)
    assert best["frames_per_tile"] in (8, 16, 32)
    assert best["threads_per_cta"] in (256, 512, 1024)
    assert best["stage_depth"] in (4, 8, 16)
    assert best["ctas_per_tile"] in (1, 2, 4, 8)
    assert best["tiles_per_item"] in (1, 2, 4)
    assert best["frames_per_lane"] in (1, 2, 4) and best["frames_per_tile"] // best["frames_per_lane"] >= 8
    assert best["sparse_frames"] in (0, 1, 2, 4, 8)
    assert ms > 0 and plan.tuning() == best
    plan.launch(ws)
    torch.cuda.synchronize()
    for g in groups:
        ref = reference(g, opts)
        assert torch.equal(g["bits"], ref["bits"]) and torch.equal(g["iters"], ref["iters"])


def test_plan_rejects_unsupported_options_and_small_workspace():
    groups = make_groups([(1024, 0.5, 4, 0.8)], seed=980)
    with pytest.raises(RuntimeError):
        q.Plan(groups, q.DecodeOpts(algo="sp_flood"))
    with pytest.raises(RuntimeError):
        q.Plan(groups, q.DecodeOpts(algo="oms_layered", prec="f16"))
    with pytest.raises(RuntimeError):
        q.Plan(groups, q.DecodeOpts(algo="oms_layered"), dict(frames_per_tile=4))
    with pytest.raises(RuntimeError):
        q.Plan(groups, q.DecodeOpts(algo="oms_layered"), dict(ctas_per_tile=3))
    with pytest.raises(RuntimeError):
        q.Plan(groups, q.DecodeOpts(algo="oms_layered"), dict(tiles_per_item=3))
    with pytest.raises(RuntimeError):          # fewer than 8 lanes per check
        q.Plan(groups, q.DecodeOpts(algo="oms_layered"), dict(frames_per_tile=8, frames_per_lane=2))
    with pytest.raises(RuntimeError):
        q.Plan(groups, q.DecodeOpts(algo="oms_layered"), dict(frames_per_lane=3))
    with pytest.raises(RuntimeError):
        q.Plan(groups, q.DecodeOpts(algo="oms_layered"), dict(sparse_frames=33))
    wide = q.Plan(groups, q.DecodeOpts(algo="oms_layered"), dict(frames_per_lane=4, threads_per_cta=1024,
                                                                 stage_depth=4))
    with pytest.raises(RuntimeError):          # four frames per lane run at most 512 threads per CTA
        wide.launch(wide.workspace())
    deep = q.Plan(groups, q.DecodeOpts(algo="oms_layered"), dict(stage_depth=16, threads_per_cta=512))
    with pytest.raises(RuntimeError):          # depth 16 runs at most 256 threads per CTA
        deep.launch(deep.workspace())
    plan = q.Plan(groups, q.DecodeOpts(algo="oms_layered"))
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError):
        plan.launch(small)
    empty = q.Plan([], q.DecodeOpts(algo="oms_layered"))
    empty.launch(empty.workspace())
    torch.cuda.synchronize()
