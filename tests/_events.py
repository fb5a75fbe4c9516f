"""Cached synthetic events for the tests (seeded; generator only, no tracking arithmetic)."""
import functools

import numpy as np

from paper_1712_09434_gb300 import synth


@functools.lru_cache(maxsize=None)
def event(name, **kw):
    makers = {
        "c1": synth.single_sector,
        "c2": synth.full_event,
        "c3": synth.central_event,
        "c5": synth.calib_event,
    }
    return synth.make_event(makers[name](**kw))


def noise_free(n_tracks=300, seed=7, theta=None, single_sector=False):
    cfg = synth.EventConfig(n_tracks=n_tracks, noise_frac=0.0, seed=seed, smear=0.0,
                            theta=theta, single_sector=single_sector)
    return synth.make_event(cfg)


def truth_hits(ev, p):
    """Clusters of generating track p in the order the particle crosses them (path length),
    approximated by (sector visit order, row) for tracks that only move outwards."""
    idx = np.nonzero(ev.mc_track == p)[0]
    return idx
