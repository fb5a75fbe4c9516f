"""Helpers that run the CUDA path through the C ABI (via the thin binding) and bring results back."""
import numpy as np
import torch

from paper_1712_09434_gb300 import capi, synth


def make_context(max_clusters, max_events=1):
    return capi.Context(max_clusters=max(int(max_clusters), 1), max_events=max_events)


def clusters_of(ev_or_batch, n_events=1):
    return capi.Clusters.from_numpy(ev_or_batch.pad_fp, ev_or_batch.time_fp, ev_or_batch.bin_off, n_events)


def run(ctx, cl, n_events=1, batch=False, stages=False, tuning=None):
    n = cl.n_clusters
    cap_t = max(n // 10 + 16, 64)
    tr = capi.Tracks(n, n_events, cap_t, max(n, 1))
    if batch:
        ctx.tpc_track_batch(cl, tr, tuning)
    else:
        ctx.tpc_track_event(cl, tr)
    st = ctx.tpc_sync_status()
    assert st == 0, capi.lib().tpc_strerror(st)
    out = tr.to_host()
    out["tracks_obj"] = tr
    if stages:
        N = max(n, 1)
        up = torch.empty(N, dtype=torch.int32, device="cuda")
        down = torch.empty(N, dtype=torch.int32, device="cuda")
        ctx.tpc_debug_copy(0, up)
        ctx.tpc_debug_copy(1, down)
        nc_t = torch.empty(1, dtype=torch.int32, device="cuda")
        ctx.tpc_debug_copy(2, nc_t)
        nc = int(nc_t.item())
        bufs = {}
        for what, name, width in [(3, "chain_start", 1), (4, "chain_len", 1), (5, "cand_n", 1),
                                  (6, "cand_slots", synth.N_ROWS), (7, "cand_rows", 1), (8, "seg_n", 1),
                                  (9, "next", 1)]:
            b = torch.empty(max(nc * width, 1), dtype=torch.int32, device="cuda")
            ctx.tpc_debug_copy(what, b)
            bufs[name] = b.cpu().numpy()[:nc * width]
        torch.cuda.synchronize()
        out.update(up=up.cpu().numpy()[:n], down=down.cpu().numpy()[:n], n_chains=nc, **bufs)
    return out


def cand_lists(out):
    """Candidate hit lists (ascending rows) from the slot representation."""
    nc = out["n_chains"]
    slots = out["cand_slots"].reshape(nc, synth.N_ROWS) if nc else np.zeros((0, synth.N_ROWS), np.int32)
    res = []
    for t in range(nc):
        r0, r1 = out["cand_rows"][t] & 0xffff, out["cand_rows"][t] >> 16
        s = slots[t, r0:r1 + 1]
        res.append(s[s >= 0])
    return res
