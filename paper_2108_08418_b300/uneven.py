"""Reverse reconciliation of an uneven batch of frames as one CUDA graph.

Each frame f has its own length n_f and SNR, hence its own quantiser range
[-4 sigma_y, 4 sigma_y], noise level sigma_n = SNR^-1/2 and per-slice code
rates (Sec. III-A: the rate of slice j follows its conditional capacity; a
slice whose rate is 0 is disclosed).  One step of the batch:

  Bob    quantise every frame with its range into m slices (Sec. III-A), then
         the syndrome of every decoded (frame, slice) with the code of its
         (n_f, rate) (Sec. II, step 5);
  Alice  for j = 0 .. m-1: the slice-j LLRs of every frame from x and the
         already reconciled slices 0..j-1 (Sec. III-B, multi-stage decoding),
         then ONE persistent plan launch decoding every frame of slice j
         (layered offset min-sum, per-frame stopping test), then the
         disclosed frames of slice j copied in the clear -- for each of the
         batch's `parts` parts (the frames of each length split between them,
         every slice of a frame in the same part) on its own stream, so the
         parts' launches overlap.

Groups of a slice's plan are runs of consecutive frames sharing (n, rate):
order the frames by (n, SNR) so that the runs are long.  All buffers are
allocated once here, so `step` allocates nothing and the whole step can be
captured in a CUDA graph (`capture`) and replayed with new x, y written into
the `x` and `y` tensors in place.
"""
from __future__ import annotations

import numpy as np

from . import DecodeOpts, Plan, qkdrec_quantise_slices_frames, qkdrec_slice_llr_frames, qkdrec_syndrome
from . import qkdrec_decode_batch, qkdrec_decode_workspace_size, qkdrec_quantise_slices, qkdrec_slice_llr
from . import quantiser_range


def _torch():
    import torch
    return torch


def frame_parts(lengths, parts: int):
    """Part of each frame: every run of consecutive frames with one length is cut
    into `parts` consecutive pieces of near-equal size (sizes differ by at most
    one frame), piece h going to part h; a run of fewer than `parts` frames
    puts its frames in distinct parts."""
    lengths = np.asarray(lengths)
    F = lengths.size
    out = np.zeros(F, dtype=np.int64)
    f = 0
    while f < F:
        g = f + 1
        while g < F and lengths[g] == lengths[f]:
            g += 1
        out[f:g] = (np.arange(g - f) * int(parts)) // (g - f)
        f = g
    return out


class UnevenBatch:
    """lengths int [F] (samples per frame, in sample order); snrs float [F];
    rates float [m][F] (0 = the slice of that frame is disclosed); codes: dict
    (n, rate) -> Code for every decoded (n_f, rates[j][f]) pair.

    decoder: None (default) decodes each slice with one persistent plan launch
    per part (layered offset min-sum, `max_iter`, `offset`); a DecodeOpts
    instead runs the plain batch decoder on every group of the slice in turn
    with those options (the same step otherwise, also capturable).
    parts: the batch's frames are split into this many parts, each decoded on
    its own stream (results do not depend on it)."""

    def __init__(self, lengths, snrs, rates, codes, m_slices: int = 5, label: str = "gray",
                 max_iter: int = 50, offset: float = 0.5, tuning: dict | None = None, device="cuda",
                 va: float = 1.0, decoder: DecodeOpts | None = None, parts: int = 2):
        torch = _torch()
        self.lengths = np.asarray(lengths, dtype=np.int64)
        self.snrs = np.asarray(snrs, dtype=np.float64)
        self.rates = np.asarray(rates, dtype=np.float64).reshape(m_slices, -1)
        F = self.F = self.lengths.size
        if self.snrs.size != F or self.rates.shape[1] != F:
            raise ValueError("lengths, snrs and rates[j] must have one entry per frame")
        self.m, self.label = int(m_slices), label
        self.device = torch.device(device)
        off = np.concatenate([[0], np.cumsum(self.lengths)]).astype(np.int64)
        self.offsets = off
        self.count = int(off[-1])
        rng = np.array([quantiser_range(s, va) for s in self.snrs], dtype=np.float64).reshape(F, 2)
        par = np.concatenate([rng, (self.snrs ** -0.5)[:, None]], axis=1)
        dev = self.device
        self.d_off = torch.from_numpy(off).to(dev)
        self.d_ranges = torch.from_numpy(np.ascontiguousarray(rng)).to(dev)
        self.d_params = torch.from_numpy(np.ascontiguousarray(par)).to(dev)
        self.x = torch.zeros(self.count, dtype=torch.float32, device=dev)
        self.y = torch.zeros(self.count, dtype=torch.float32, device=dev)
        self.bob = torch.zeros((self.m, self.count), dtype=torch.uint8, device=dev)
        self.alice = torch.zeros((self.m, self.count), dtype=torch.uint8, device=dev)
        self.llr = torch.zeros(self.count, dtype=torch.float32, device=dev)
        self.iters = torch.zeros((self.m, F), dtype=torch.int32, device=dev)
        self.conv = torch.ones((self.m, F), dtype=torch.uint8, device=dev)
        self.opts = DecodeOpts(algo="oms_layered", prec="f32", max_iter=max_iter, offset=offset, early_stop=True)
        self.group_opts = decoder
        self.codes = codes
        # Frames are cut into `parts` parts -- the frames of each length split
        # into consecutive pieces, one per part, the same for every slice (a
        # frame's slices all decode in its part, each after its lower slices):
        # the parts are independent reconciliations, decoded on their own
        # streams, so one part's slice launch fills the SMs another part's
        # launch frees at its end.  Per part and slice: groups (runs of frames
        # with one code), disclosed sample ranges, the frame runs that need
        # slice-j LLRs.
        self.parts = max(1, int(parts))
        part_of = self.part_of = frame_parts(self.lengths, self.parts)
        self.groups = [[] for _ in range(self.m)]
        self.disclosed = [[] for _ in range(self.m)]
        self.synd = []
        self._parts = [dict(groups=[[] for _ in range(self.m)], disclosed=[[] for _ in range(self.m)],
                            llr_runs=[[] for _ in range(self.m)], plans=[]) for _ in range(self.parts)]
        for j in range(self.m):
            pieces = []                     # (part, first frame, end frame, code or None)
            f = 0
            while f < F:
                key = (int(self.lengths[f]), float(self.rates[j, f]), int(part_of[f]))
                g = f + 1
                while g < F and (int(self.lengths[g]), float(self.rates[j, g]), int(part_of[g])) == key:
                    g += 1
                if key[1] > 0 and key[:2] not in codes:
                    raise KeyError(f"no code for (n, rate) = {key[:2]}")
                pieces.append((key[2], f, g, codes[key[:2]] if key[1] > 0 else None))
                f = g
            total = sum((g - f) * c.M for _, f, g, c in pieces if c is not None)
            synd = torch.zeros(max(total, 1), dtype=torch.uint8, device=dev)
            so = 0
            for h, f, g, c in pieces:
                P = self._parts[h]
                a, b = int(off[f]), int(off[g])
                if c is None:
                    self.disclosed[j].append((a, b))
                    P["disclosed"][j].append((a, b))
                    continue
                nf = g - f
                gd = dict(code=c, f0=f, f1=g, a=a, b=b,
                          llr=self.llr[a:b].view(nf, c.n), bits=self.alice[j, a:b].view(nf, c.n),
                          synd=synd[so:so + nf * c.M].view(nf, c.M),
                          iters=self.iters[j, f:g], conv=self.conv[j, f:g])
                so += nf * c.M
                self.groups[j].append(gd)
                P["groups"][j].append(gd)
                runs_j = P["llr_runs"][j]            # frames of this part that need slice-j LLRs
                if runs_j and runs_j[-1][1] == f:
                    runs_j[-1][1] = g
                else:
                    runs_j.append([f, g])
            self.synd.append(synd)
        self.plans = []
        sizes = []
        for P in self._parts:
            if decoder is None:
                P["plans"] = [Plan(P["groups"][j], self.opts, tuning) for j in range(self.m)]
                self.plans += P["plans"]
                sizes.append(max(p.workspace_size() for p in P["plans"]))
            else:
                sizes.append(max([qkdrec_decode_workspace_size(g["code"], g["f1"] - g["f0"], decoder)
                                  for gs in P["groups"] for g in gs] or [1]))
        # one workspace, a 256-byte-aligned piece per part
        offs = np.concatenate([[0], np.cumsum([(sz + 255) // 256 * 256 for sz in sizes])])
        self.ws = torch.empty(max(int(offs[-1]), 256), dtype=torch.uint8, device=dev)
        self._ws = [self.ws[int(offs[h]):int(offs[h]) + sizes[h]] for h in range(self.parts)]
        self.graph = None
        self._side = torch.cuda.Stream(dev)
        self._pstreams = [torch.cuda.Stream(dev) for _ in range(self.parts - 1)]
        self._synd_done = [torch.cuda.Event() for _ in range(self.m)]

    # ------------------------------------------------------------------ run
    def step(self, overlap: bool = True):
        """Enqueue one reconciliation of the batch in `x`, `y` on the current stream.

        Bob's syndromes depend only on his slices, so they run on a side stream
        (forked after the quantiser) while Alice decodes; each part of the batch
        runs its slices in order on its own stream (the first on the current
        one), its decode of slice j waiting only for the syndromes of slice j;
        every stream is joined back before the step ends.  overlap=False runs
        the same work in order on the current stream alone (for timing each
        kernel by itself)."""
        torch = _torch()
        main = torch.cuda.current_stream(self.device)
        qkdrec_quantise_slices_frames(self.y, self.d_off, self.d_ranges, self.m, self.label, want_idx=False,
                                      bits_out=self.bob)
        side = self._side if overlap else main
        pstreams = self._pstreams if overlap else [main] * len(self._pstreams)
        side.wait_stream(main)
        for st in pstreams:
            st.wait_stream(main)
        with torch.cuda.stream(side):
            for j in range(self.m):
                for g in self.groups[j]:
                    nf, n = g["f1"] - g["f0"], g["code"].n
                    qkdrec_syndrome(g["code"], self.bob[j, g["a"]:g["b"]].view(nf, n), out=g["synd"])
                self._synd_done[j].record(side)
        for h, P in enumerate(self._parts):
            st = main if h == 0 else pstreams[h - 1]
            with torch.cuda.stream(st):
                for j in range(self.m):
                    self._llr(P, j)
                    st.wait_event(self._synd_done[j])
                    if self.group_opts is not None:
                        for g in P["groups"][j]:
                            qkdrec_decode_batch(g["code"], g["llr"], g["synd"], self.group_opts,
                                                workspace=self._ws[h],
                                                out=dict(bits=g["bits"], iters=g["iters"], converged=g["conv"]))
                    elif P["groups"][j]:
                        P["plans"][j].launch(self._ws[h])
                    for a, b in P["disclosed"][j]:
                        self.alice[j, a:b].copy_(self.bob[j, a:b])
        for st in pstreams:
            main.wait_stream(st)
        main.wait_stream(side)

    def _llr(self, P, j):
        """Slice-j LLRs of the frames of part P that decode slice j."""
        for f, g in P["llr_runs"][j]:
            qkdrec_slice_llr_frames(self.x, self.d_off[f:g + 1], self.d_params[f:g], self.m, j,
                                    self.alice[:j] if j else None, self.label, out=self.llr)

    def autotune(self, max_iter: int = 10):
        """Pick each plan's fastest tuning (per part and slice, part-major) on the
        batch now in x, y (synchronous)."""
        torch = _torch()
        out = []
        if self.group_opts is not None:
            return [(None, 0.0)] * self.m
        self.step()
        torch.cuda.synchronize(self.device)
        for h, P in enumerate(self._parts):
            for j, p in enumerate(P["plans"]):
                # the plan decodes the LLRs of slice j: recompute them first
                self._llr(P, j)
                if not P["groups"][j]:
                    out.append((None, 0.0))
                    continue
                out.append(p.autotune(self._ws[h], max_iter))
                p.launch(self._ws[h])
        torch.cuda.synchronize(self.device)
        self.graph = None
        return out

    def capture(self):
        """Capture `step` in a CUDA graph (after one eager step that sets kernel attributes)."""
        torch = _torch()
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.step()
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        return self.graph

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    # --------------------------------------------------------------- results
    def frame_ok(self):
        """bool [m][F]: Alice's slice equals Bob's (disclosed slices count as equal)."""
        torch = _torch()
        ok = torch.ones((self.m, self.F), dtype=torch.bool, device=self.device)
        f = 0
        while f < self.F:                       # runs of frames with one length
            n = int(self.lengths[f])
            g = f + 1
            while g < self.F and int(self.lengths[g]) == n:
                g += 1
            a, b = int(self.offsets[f]), int(self.offsets[g])
            if n > 0:
                ok[:, f:g] = (self.alice[:, a:b] == self.bob[:, a:b]).view(self.m, g - f, n).all(dim=2)
            f = g
        return ok

    def reconciled_bits(self):
        """Bits of decoded (non-disclosed) slices in frames reconciled correctly."""
        ok = self.frame_ok().cpu().numpy()
        dec = self.rates > 0
        return int(np.sum(ok * dec * self.lengths[None, :]))

    def decoded_bits(self):
        return int(np.sum((self.rates > 0) * self.lengths[None, :]))

    def destroy(self):
        for p in self.plans:
            p.destroy()
        self.plans = []
        self.graph = None


# ------------------------------------------------------------- rate back-off
def backoff_rates(points, start_rate, codes_for, sample, trial_frames: int = 32, max_fail: int = 1,
                  step: float = 3 / 64, min_rate: float = 0.10, m_slices: int = 5, label: str = "gray",
                  max_iter: int = 50, offset: float = 0.5, tuning: dict | None = None, device="cuda",
                  va: float = 1.0):
    """Code-rate back-off on trial frames (Sec. V-B: pick the rate closest to
    capacity, test whether the code fails too often, else lower the rate by a
    fixed step and test again).

    points      list of (n, snr, j): block length, SNR, slice
    start_rate  dict point -> first rate tried (on the 1/64 grid)
    codes_for   callable: set of (n, rate) -> dict (n, rate) -> Code
    sample      callable: point -> (x, y) float32 arrays of trial_frames * n samples
    Each point's trial frames are quantised and their slice-j LLRs formed with
    Bob's own lower slices (lower slices reconciled); every round decodes all
    pending points in one plan launch (layered offset min-sum) and lowers the
    rate of each point with more than `max_fail` frame errors by `step`
    (rounded to 1/64).  A rate below `min_rate` means the slice is disclosed.
    Returns dict point -> (rate, frame errors of the accepted rate); rate 0.0
    = disclosed.
    """
    torch = _torch()
    dev = torch.device(device)
    opts = DecodeOpts(algo="oms_layered", prec="f32", max_iter=max_iter, offset=offset, early_stop=True)
    trial = {}
    for p in points:
        n, snr, j = p
        x, y = sample(p)
        lo, hi = quantiser_range(snr, va)
        xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(dev)
        yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).to(dev)
        _, bits = qkdrec_quantise_slices(yd, m_slices, lo, hi, label, want_idx=False)
        llr = qkdrec_slice_llr(xd, m_slices, j, lo, hi, snr ** -0.5, bits[:j] if j else None, label)
        trial[p] = (llr.view(trial_frames, n), bits[j].reshape(trial_frames, n).contiguous())
    rate = {p: float(start_rate[p]) for p in points}
    done = {}
    for p in points:
        if rate[p] < min_rate:
            done[p] = (0.0, 0)
    pending = [p for p in points if p not in done]
    while pending:
        codes = codes_for({(p[0], rate[p]) for p in pending})
        groups = []
        for p in pending:
            c = codes[(p[0], rate[p])]
            llr, bob = trial[p]
            groups.append(dict(code=c, llr=llr, synd=qkdrec_syndrome(c, bob),
                               bits=torch.empty_like(bob),
                               iters=torch.empty(trial_frames, dtype=torch.int32, device=dev),
                               conv=torch.empty(trial_frames, dtype=torch.uint8, device=dev)))
        plan = Plan(groups, opts, tuning)
        plan.launch(plan.workspace(dev))
        torch.cuda.synchronize(dev)
        fails = [int((g["bits"] != trial[p][1]).any(dim=1).sum().item()) for p, g in zip(pending, groups)]
        plan.destroy()
        nxt = []
        for p, f in zip(pending, fails):
            if f <= max_fail:
                done[p] = (rate[p], f)
                continue
            r = np.floor((rate[p] - step) * 64 + 0.5) / 64
            if r < min_rate:
                done[p] = (0.0, f)
            else:
                rate[p] = float(r)
                nxt.append(p)
        pending = nxt
    return done
