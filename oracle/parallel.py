"""All-core driver of the FP64 oracle (test infrastructure: the CPU baseline's multi-threaded
timing and the benchmark's accuracy sample; the product never imports it).

The arithmetic is the oracle's own C routines, unchanged; only the work is split: the
projection and its reverse mode over ranges of Gaussians, the compositing and its reverse mode
over ranges of tiles (tiles are independent, Sec. 3's compositing is per pixel). Threads that
accumulate do so into buffers of their own, summed at the end, so gradient sums are taken in a
different order than the single-threaded oracle's (the last bits of float64 may differ).
ctypes releases the GIL for the duration of each C call, so Python threads run the C code
concurrently. The binning of a view is split into bands of tile rows, each sorted on its own
thread; the bands concatenated in row order are the view's sorted pairs.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from typing import List

import numpy as np

from . import (C, LOWPASS, N_MARGINS, Bins, Composed, Projected, _grad_params, _p, _project_backward,
               decision_inputs, lib, project)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _chunks(n: int, k: int) -> List[tuple]:
    k = max(1, min(k, n)) if n > 0 else 1
    edges = np.linspace(0, n, k + 1).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def _sub(comp: Composed, a: int, b: int) -> Composed:
    return Composed(*(x[a:b] for x in comp.arrays()), model_id=comp.model_id[a:b], n_models=comp.n_models,
                    sh=None if comp.sh is None else comp.sh[a:b], sh_degree=comp.sh_degree)


def project_parallel(pool, comp: Composed, table, cam, threads: int, lowpass: float = LOWPASS) -> Projected:
    parts = list(pool.map(lambda ab: project(_sub(comp, *ab), table, cam, lowpass), _chunks(comp.n, threads)))
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])
    return Projected(uv=cat("uv"), cov=cat("cov"), conic=cat("conic"), opacity=cat("opacity"), rgb=cat("rgb"),
                     depth=cat("depth"), radius=cat("radius"), radius_margin=cat("radius_margin"),
                     depth_margin=cat("depth_margin"))


def bin_view_parallel(pool, p: Projected, cam, threads: int, tile=(16, 16)) -> Bins:
    """The binning of one view (what bin_pairs gives for it) from bands of tile rows, each
    sorted on its own thread (orc_bin_view_rows), concatenated in row order."""
    uv32, rad, d32 = (np.ascontiguousarray(a[0]) for a in decision_inputs([p]))
    gx, gy = (cam.W + tile[0] - 1) // tile[0], (cam.H + tile[1] - 1) // tile[1]

    def band(rows):
        args = (C.c_int64(len(rad)), _p(uv32, C.c_float), _p(rad, C.c_int32), _p(d32, C.c_float), C.c_int32(cam.W),
                C.c_int32(cam.H), C.c_int32(tile[0]), C.c_int32(tile[1]), C.c_int64(0), C.c_int32(rows[0]),
                C.c_int32(rows[1]))
        dk, dv = np.zeros(1, np.uint64), np.zeros(1, np.uint32)
        cnt = lib().orc_bin_view_rows(*args, _p(dk, C.c_uint64), _p(dv, C.c_uint32), C.c_int64(0))
        keys, vals = np.zeros(max(cnt, 1), np.uint64), np.zeros(max(cnt, 1), np.uint32)
        lib().orc_bin_view_rows(*args, _p(keys, C.c_uint64), _p(vals, C.c_uint32), C.c_int64(cnt))
        return keys[:cnt], vals[:cnt]
    parts = list(pool.map(band, _chunks(gy, 4 * threads)))
    keys = np.concatenate([k for k, _ in parts]) if parts else np.zeros(0, np.uint64)
    vals = np.concatenate([v for _, v in parts]) if parts else np.zeros(0, np.uint32)
    t = (keys >> np.uint64(32)).astype(np.int64)
    nt = gx * gy
    ranges = np.zeros((nt, 2), np.uint32)
    ranges[:, 0] = np.searchsorted(t, np.arange(nt), side="left")
    ranges[:, 1] = np.searchsorted(t, np.arange(nt), side="right")
    ranges[ranges[:, 0] == ranges[:, 1]] = 0  # empty tiles: [0, 0), as orc_bin leaves them
    return Bins(keys=keys, values=vals, ranges=ranges, tile_offset=np.array([0, nt], np.int64))


def render_view_parallel(comp: Composed, table, cam, bg, threads: int = 0, tile=(16, 16), lowpass: float = LOWPASS):
    """Forward of one view on all cores: (rgba [H, W, 4], final T, last, margins, projection, bins)."""
    threads = threads or default_threads()
    bg = np.ascontiguousarray(bg, np.float64)
    with ThreadPoolExecutor(threads) as pool:
        p = project_parallel(pool, comp, table, cam, threads, lowpass)
        bins = bin_view_parallel(pool, p, cam, threads, tile)
        rgba = np.zeros((cam.H, cam.W, 4)); T = np.zeros((cam.H, cam.W))
        last = np.zeros((cam.H, cam.W), np.uint32); mg = np.zeros((cam.H, cam.W, N_MARGINS))
        nt = ((cam.W + tile[0] - 1) // tile[0]) * ((cam.H + tile[1] - 1) // tile[1])

        def run(ab):  # disjoint tiles write disjoint pixels
            lib().orc_render_view_tiles(_p(p.uv), _p(p.conic), _p(p.opacity), _p(p.rgb),
                                        _p(bins.values, C.c_uint32), _p(bins.ranges, C.c_uint32), C.c_int64(0),
                                        C.c_int32(cam.W), C.c_int32(cam.H), C.c_int32(tile[0]), C.c_int32(tile[1]),
                                        _p(bg), _p(rgba), _p(T), _p(last, C.c_uint32), _p(mg), C.c_int64(ab[0]),
                                        C.c_int64(ab[1]))
        list(pool.map(run, _chunks(nt, 4 * threads)))
    return rgba, T, last, mg, p, bins


def render_backward_view_parallel(comp: Composed, table, cam, p: Projected, bins, dL_drgba, bg, threads: int = 0,
                                  tile=(16, 16), lowpass: float = LOWPASS):
    """Reverse mode of one view on all cores: (parameter gradients, edit-table gradient, light gradient)."""
    threads = threads or default_threads()
    bg = np.ascontiguousarray(bg, np.float64)
    d = np.ascontiguousarray(dL_drgba, np.float64)
    n = comp.n
    nt = ((cam.W + tile[0] - 1) // tile[0]) * ((cam.H + tile[1] - 1) // tile[1])
    with ThreadPoolExecutor(threads) as pool:
        def blend(ab):
            g = dict(uv=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)))
            lib().orc_render_view_backward_tiles(_p(p.uv), _p(p.conic), _p(p.opacity), _p(p.rgb),
                                                 _p(bins.values, C.c_uint32), _p(bins.ranges, C.c_uint32),
                                                 C.c_int64(0), C.c_int32(cam.W), C.c_int32(cam.H), C.c_int32(tile[0]),
                                                 C.c_int32(tile[1]), _p(bg), _p(d), _p(g["uv"]), _p(g["conic"]),
                                                 _p(g["opacity"]), _p(g["rgb"]), C.c_int64(ab[0]), C.c_int64(ab[1]))
            return g
        parts = list(pool.map(blend, _chunks(nt, threads)))
        g = {k: np.sum([q[k] for q in parts], axis=0) for k in parts[0]}
        params = _grad_params(comp)

        def chain(ab):  # disjoint Gaussians write disjoint parameter gradients; edits per thread
            a, b = ab
            de = np.zeros_like(table)
            dl = np.zeros(3)
            sub_p = {k: v[a:b] for k, v in params.items()}
            sub_g = {k: np.ascontiguousarray(v[a:b]) for k, v in g.items()}
            _project_backward(_sub(comp, a, b), table, cam, lowpass, sub_g, sub_p, de, dl)
            return de, dl
        outs = list(pool.map(chain, _chunks(n, threads)))
    return params, np.sum([o[0] for o in outs], axis=0), np.sum([o[1] for o in outs], axis=0)


__all__ = ["default_threads", "project_parallel", "bin_view_parallel", "render_view_parallel",
           "render_backward_view_parallel"]
