"""Per-iteration metrics of a ForceAtlas2 run as JSON lines.

A long layout of one component (Section 3.2) is advanced through the
library's resumable session (bgl_fa2_session_*) in chunks of iterations.
After each chunk every iteration of it becomes one JSON object on its own
line:

  {"component": c, "n": n_c, "iter": k, "swing": swg_k, "traction": trc_k,
   "s_G": s_G_k, "ms": t, "chunk": m}

k counts the iterations run on the session so far (1 for the first);
swing, traction and s_G are the values the device computed in iteration k
(returned by bgl_fa2_session_advance); t is the wall time of the chunk of m
iterations that held k, divided evenly among them -- a chunk runs as one
graph launch, so there is no finer time without slowing the iterations.
This is host-side logging of the library's own numbers: it computes
nothing of the method.  The final positions are bitwise those of one
bgl_fa2_step call with the same number of iterations.
"""
from __future__ import annotations

import json
import time


def run_logged(graph, c: int, p, iters: int, xy=None, out=None, chunk: int = 50, resume: bool = False,
               clock=time.perf_counter):
    """Runs `iters` ForceAtlas2 iterations on component c of `graph` and
    writes one JSON line per iteration to `out` (a path or a text stream).

    xy: the component's local start positions (n_c x 2); ignored with
    resume=True, which continues the graph's current session (for example
    one restored by state_load; c must be its component) and numbers its
    iterations on from the ones it has run.  chunk: iterations per session
    call.  Returns the positions after the last iteration (n_c x 2, FP32)."""
    if chunk < 1:
        raise ValueError("chunk must be >= 1")
    if iters < 0:
        raise ValueError("iters must be >= 0")
    if resume:
        coff = graph.component_nodes()[0]
        n = int(coff[c + 1] - coff[c])
        _, done = graph.session_positions(n)
    else:
        if xy is None:
            raise ValueError("xy is required unless resume=True")
        n = len(xy)
        graph.session_begin(c, p, xy)
        done = 0
    own = isinstance(out, str)
    f = open(out, "w") if own else out
    try:
        left = iters
        while left > 0:
            m = min(chunk, left)
            t0 = clock()
            stats = graph.session_advance(m)
            ms = (clock() - t0) * 1e3 / m
            for j in range(m):
                rec = {"component": int(c), "n": int(n), "iter": done + j + 1, "swing": float(stats[j][0]),
                       "traction": float(stats[j][1]), "s_G": float(stats[j][2]), "ms": ms, "chunk": m}
                if f is not None:
                    f.write(json.dumps(rec) + "\n")
            if f is not None:
                f.flush()
            done += m
            left -= m
    finally:
        if own:
            f.close()
    xy_out, _ = graph.session_positions(n)
    return xy_out


def read(path):
    """The records of a metrics file, in order."""
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]
