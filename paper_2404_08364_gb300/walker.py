"""Torch-facing wrapper of the C ABI: device memory and streams come from
PyTorch, every walk step runs in libfw.so.

    g = DeviceGraph.from_graph(fw_inputs.rmat(20), device="cuda")
    paths, plen = g.walk("node2vec", starts, max_len=80, seed=42, mode="fast", p=2, q=0.5)
"""

from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from . import _fw

_P = ctypes.c_void_p


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else _P(t.data_ptr())


def _i32(t, device):
    if t is None:
        return None
    t = torch.as_tensor(t)
    if t.dtype != torch.int32:
        t = t.to(torch.int32)
    return t.to(device).contiguous()


def _stream_handle(stream) -> Optional[_P]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return _P(stream.cuda_stream)


class DeviceGraph:
    """A CSR graph resident on one GPU, owned by the library (or borrowed)."""

    def __init__(self, handle: _P, n: int, m: int, keep=()):
        self._h = handle
        self.n, self.m = n, m
        self._keep = keep  # borrowed tensors stay alive with the graph

    @classmethod
    def from_tensors(cls, row_ptr, col, w_f32=None, w_u32=None, etype=None, borrow=False,
                     validate=True, device="cuda") -> "DeviceGraph":
        L = _fw.lib()
        dev = torch.device(device)
        ts = []
        for t, dt in ((row_ptr, torch.int64), (col, torch.int32), (w_f32, torch.float32),
                      (w_u32, torch.int32), (etype, torch.int8)):
            if t is None:
                ts.append(None)
                continue
            t = torch.as_tensor(t)
            if t.dtype != dt:
                t = t.view(dt) if t.element_size() == torch.empty(0, dtype=dt).element_size() else t.to(dt)
            ts.append(t.to(dev).contiguous())
        n = ts[0].numel() - 1
        m = ts[1].numel()
        flags = (_fw.FW_BORROW if borrow else _fw.FW_DEVICE_PTRS) | (0 if validate else _fw.FW_NO_VALIDATE)
        h = _P()
        with torch.cuda.device(dev):
            _fw.check(L.fw_load_csr(ctypes.byref(h), n, m, *[_ptr(t) for t in ts], flags))
        return cls(h, n, m, keep=tuple(ts) if borrow else ())

    @classmethod
    def from_graph(cls, g, device="cuda", borrow=False, validate=True) -> "DeviceGraph":
        return cls.from_tensors(g.row_ptr, g.col, g.w_f32, g.w_u32, g.etype, borrow=borrow,
                                validate=validate, device=device)

    # ------------------------------------------------------------------ walks
    def walk(self, algo, starts, max_len: int, seed: int, mode="exact", p=1.0, q=1.0, scale=2,
             schema: Sequence[int] = (0, 1, 2, 3, 4), ppr_stop=0.2, lengths=None, prev=None, step0=None,
             q_id0: int = 0, paths=None, path_len=None, stream=None):
        """Run one batch of walks; returns (paths [n_q, max_len+1] int32, path_len [n_q] int32).

        Tensors on the GPU are used in place; CPU tensors are staged by the
        library (the call then returns with the results on the host)."""
        algo = _fw.ALGOS.get(algo, algo)
        prm = _fw.make_params(mode, p, q, scale, schema, ppr_stop)
        st = torch.as_tensor(starts)
        dev = st.device
        st = _i32(st, dev)
        n_q = st.numel()
        if paths is None:
            paths = torch.empty((n_q, max_len + 1), dtype=torch.int32, device=dev)
        if path_len is None:
            path_len = torch.empty(n_q, dtype=torch.int32, device=dev)
        ln, pv, s0 = _i32(lengths, dev), _i32(prev, dev), _i32(step0, dev)
        sh = _stream_handle(stream) if dev.type == "cuda" else None
        _fw.check(_fw.lib().fw_walk_ex(self._h, algo, ctypes.byref(prm), _ptr(st), n_q, _ptr(ln), max_len,
                                       seed & 0xFFFFFFFFFFFFFFFF, q_id0, _ptr(pv), _ptr(s0), _ptr(paths),
                                       _ptr(path_len), sh))
        return paths, path_len

    def walk_batched(self, algo, starts, max_len: int, seed: int, mode="exact", p=1.0, q=1.0, scale=2,
                     schema: Sequence[int] = (0, 1, 2, 3, 4), ppr_stop=0.2, lengths=None, q_id0: int = 0,
                     budget_bytes: int = 0, paths=None, path_len=None):
        """Walks whose results may exceed device memory (fw_walk_batched):
        host inputs and outputs, batches of Eq. 3's size on two streams.
        Returns (paths, path_len, queries per batch); outputs are pinned host
        tensors unless given."""
        algo = _fw.ALGOS.get(algo, algo)
        prm = _fw.make_params(mode, p, q, scale, schema, ppr_stop)
        st = _i32(torch.as_tensor(starts), "cpu")
        n_q = st.numel()
        if paths is None:
            paths = torch.empty((n_q, max_len + 1), dtype=torch.int32).pin_memory()
        if path_len is None:
            path_len = torch.empty(n_q, dtype=torch.int32).pin_memory()
        ln = _i32(lengths, "cpu")
        bq = ctypes.c_int64()
        _fw.check(_fw.lib().fw_walk_batched(self._h, algo, ctypes.byref(prm), _ptr(st), n_q, _ptr(ln), max_len,
                                            seed & 0xFFFFFFFFFFFFFFFF, q_id0, int(budget_bytes), _ptr(paths),
                                            _ptr(path_len), ctypes.byref(bq)))
        return paths, path_len, bq.value

    def _requests(self, requests):
        arr = (_fw.Request * len(requests))()
        outs, keep = [], []
        for i, r in enumerate(requests):
            st = _i32(r["starts"], "cuda")
            n_q = st.numel()
            L = int(r["max_len"])
            paths = r.get("paths")
            if paths is None:
                paths = torch.empty((n_q, L + 1), dtype=torch.int32, device=st.device)
            plen = r.get("path_len")
            if plen is None:
                plen = torch.empty(n_q, dtype=torch.int32, device=st.device)
            ln, pv, s0 = (_i32(r.get(k), st.device) for k in ("lengths", "prev", "step0"))
            keep += [st, ln, pv, s0]
            q = arr[i]
            q.algo = _fw.ALGOS.get(r["algo"], r["algo"])
            q.params = _fw.make_params(r.get("mode", "exact"), r.get("p", 1.0), r.get("q", 1.0),
                                       r.get("scale", 2), r.get("schema", (0, 1, 2, 3, 4)),
                                       r.get("ppr_stop", 0.2))
            q.starts, q.n_q, q.max_len = st.data_ptr(), n_q, L
            q.lengths = ln.data_ptr() if ln is not None else None
            q.prev = pv.data_ptr() if pv is not None else None
            q.step0 = s0.data_ptr() if s0 is not None else None
            q.seed = int(r["seed"]) & 0xFFFFFFFFFFFFFFFF
            q.q_id0 = int(r.get("q_id0", 0))
            q.paths, q.path_len = paths.data_ptr(), plen.data_ptr()
            outs.append((paths, plen))
        return arr, outs, keep

    def walk_noalloc(self, requests, stream=None):
        """Like walk_multi, through fw_walk_noalloc: the library allocates no
        device memory for the launch (up to 1024 requests, device tensors)."""
        arr, outs, keep = self._requests(requests)
        _fw.check(_fw.lib().fw_walk_noalloc(self._h, arr, len(requests), _stream_handle(stream)))
        return outs

    def walk_multi(self, requests, stream=None):
        """requests: list of dicts with keys algo, starts, max_len, seed, mode,
        p, q, scale, schema, ppr_stop, lengths, prev, step0, q_id0, paths,
        path_len (device tensors).  One launch for all; returns the list of
        (paths, path_len)."""
        arr = (_fw.Request * len(requests))()
        outs, keep = [], []
        for i, r in enumerate(requests):
            st = _i32(r["starts"], "cuda")
            n_q = st.numel()
            L = int(r["max_len"])
            paths = r.get("paths")
            if paths is None:
                paths = torch.empty((n_q, L + 1), dtype=torch.int32, device=st.device)
            plen = r.get("path_len")
            if plen is None:
                plen = torch.empty(n_q, dtype=torch.int32, device=st.device)
            ln, pv, s0 = (_i32(r.get(k), st.device) for k in ("lengths", "prev", "step0"))
            keep += [st, ln, pv, s0]
            q = arr[i]
            q.algo = _fw.ALGOS.get(r["algo"], r["algo"])
            q.params = _fw.make_params(r.get("mode", "exact"), r.get("p", 1.0), r.get("q", 1.0),
                                       r.get("scale", 2), r.get("schema", (0, 1, 2, 3, 4)),
                                       r.get("ppr_stop", 0.2))
            q.starts, q.n_q, q.max_len = st.data_ptr(), n_q, L
            q.lengths = ln.data_ptr() if ln is not None else None
            q.prev = pv.data_ptr() if pv is not None else None
            q.step0 = s0.data_ptr() if s0 is not None else None
            q.seed = int(r["seed"]) & 0xFFFFFFFFFFFFFFFF
            q.q_id0 = int(r.get("q_id0", 0))
            q.paths, q.path_len = paths.data_ptr(), plen.data_ptr()
            outs.append((paths, plen))
        _fw.check(_fw.lib().fw_walk_multi(self._h, arr, len(requests), _stream_handle(stream)))
        return outs

    def capture_multi(self, requests) -> "Exec":
        """Record the multi-request launch into a CUDA graph (fw_capture_multi);
        replay it with Exec.launch().  The request tensors stay attached to it."""
        arr, outs, keep = self._requests(requests)
        h = _P()
        _fw.check(_fw.lib().fw_capture_multi(self._h, arr, len(requests), ctypes.byref(h)))
        return Exec(h, outs, keep)

    def autotune(self, requests, reps: int = 2) -> dict:
        """Pick the engine tuning on a sample workload (fw_autotune); returns it
        with the measured steps/s (0 on a cache hit)."""
        arr, outs, keep = self._requests(requests)
        t = _fw.Tuning()
        rate = ctypes.c_double()
        _fw.check(_fw.lib().fw_autotune(self._h, arr, len(requests), int(reps), ctypes.byref(t), ctypes.byref(rate)))
        d = {k: getattr(t, k) for k, _ in _fw.Tuning._fields_}
        d["steps_per_s"] = rate.value
        return d

    # ------------------------------------------------------------ management
    def set_tuning(self, block_threads=0, slots=0, d_warp=0, ctas_per_sm=0):
        t = _fw.Tuning(block_threads, slots, d_warp, ctas_per_sm)
        _fw.check(_fw.lib().fw_set_tuning(self._h, ctypes.byref(t)))

    def get_tuning(self) -> dict:
        t = _fw.Tuning()
        _fw.check(_fw.lib().fw_get_tuning(self._h, ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in _fw.Tuning._fields_}

    def stats(self) -> dict:
        s = _fw.Stats()
        _fw.check(_fw.lib().fw_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _fw.Stats._fields_}

    def stats_reset(self, stream=None):
        _fw.check(_fw.lib().fw_stats_reset(self._h, _stream_handle(stream)))

    def info(self) -> dict:
        n, m, dm = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _fw.check(_fw.lib().fw_graph_info(self._h, *(ctypes.byref(x) for x in (n, m, dm, a, b, c))))
        return {"n": n.value, "m": m.value, "d_max": dm.value, "has_f32": bool(a.value),
                "has_u32": bool(b.value), "has_type": bool(c.value)}

    def free(self):
        if self._h:
            _fw.lib().fw_free(self._h)
            self._h = None
            self._keep = ()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Exec:
    """A captured multi-request launch (CUDA graph)."""

    def __init__(self, handle, outs, keep):
        self._h = handle
        self.outputs = outs
        self._keep = keep

    def launch(self, stream=None):
        _fw.check(_fw.lib().fw_exec_launch(self._h, _stream_handle(stream)))
        return self.outputs

    def close(self):
        if self._h:
            _fw.lib().fw_exec_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Served form (fw_server_*): a resident graph, requests admitted by
    output-arena memory and run by the persistent engine as they arrive.

        srv = Server(dg, mode="fast", mem_budget=1 << 30)
        t = srv.submit("node2vec", starts_cpu, max_len=80, seed=7, p=2, q=0.5)
        paths, plen, latency_s = srv.result(t)
    """

    def __init__(self, graph: DeviceGraph, mode="fast", mem_budget: int = 1 << 30, max_requests: int = 1024,
                 idle_ms: float = 20.0):
        self._g = graph
        self.mode = _fw.MODES.get(mode, mode)
        h = _P()
        _fw.check(_fw.lib().fw_server_create(graph._h, self.mode, int(mem_budget), int(max_requests),
                                             float(idle_ms), ctypes.byref(h)))
        self._h = h
        self._out = {}

    def submit(self, algo, starts, max_len: int, seed: int, p=1.0, q=1.0, scale=2,
               schema: Sequence[int] = (0, 1, 2, 3, 4), ppr_stop=0.2, lengths=None, prev=None, step0=None,
               q_id0: int = 0) -> int:
        """Queue one request (host tensors); returns its ticket."""
        st = _i32(starts, "cpu")
        n_q = st.numel()
        paths = torch.empty((n_q, max_len + 1), dtype=torch.int32).pin_memory()
        plen = torch.empty(n_q, dtype=torch.int32).pin_memory()
        ln, pv, s0 = _i32(lengths, "cpu"), _i32(prev, "cpu"), _i32(step0, "cpu")
        r = _fw.Request()
        r.algo = _fw.ALGOS.get(algo, algo)
        r.params = _fw.make_params(self.mode, p, q, scale, schema, ppr_stop)
        r.starts, r.n_q, r.max_len = st.data_ptr(), n_q, int(max_len)
        r.lengths = ln.data_ptr() if ln is not None else None
        r.prev = pv.data_ptr() if pv is not None else None
        r.step0 = s0.data_ptr() if s0 is not None else None
        r.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        r.q_id0 = int(q_id0)
        r.paths, r.path_len = paths.data_ptr(), plen.data_ptr()
        t = ctypes.c_uint64()
        _fw.check(_fw.lib().fw_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._out[t.value] = (paths, plen)
        return t.value

    def poll(self, ticket: int):
        done, lat = ctypes.c_int32(), ctypes.c_double()
        _fw.check(_fw.lib().fw_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(lat)))
        return done.value, lat.value

    def result(self, ticket: int, timeout_s: float = 120.0):
        """Wait for a ticket; returns (paths, path_len, latency_s) and forgets it."""
        lat = ctypes.c_double()
        _fw.check(_fw.lib().fw_server_wait(self._h, ticket, float(timeout_s), ctypes.byref(lat)))
        _fw.check(_fw.lib().fw_server_release(self._h, ticket))
        paths, plen = self._out.pop(ticket)
        return paths, plen, lat.value

    def stats(self) -> dict:
        s = _fw.ServerStats()
        _fw.check(_fw.lib().fw_server_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _fw.ServerStats._fields_}

    def close(self):
        if self._h:
            _fw.lib().fw_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SAMPLERS = {"expj": 0, "dprs": 1, "zprs": 2}


def sample(method: str, weights, reps: int, seed: int = 1, width: int = 32, out=None, stream=None, timed=True):
    """reps independent weighted draws from one weight vector (fw_sampler_run):
    method "expj" (the engine's reservoir), "dprs" (Alg. 3) or "zprs"
    (Alg. 4), by groups of `width` threads (32 or 256).  weights: float32
    CUDA tensor.  Returns (indices int32 CUDA tensor, launch ms or None)."""
    w = weights.contiguous()
    if w.dtype != torch.float32 or w.device.type != "cuda":
        raise ValueError("weights must be a float32 CUDA tensor")
    if out is None:
        out = torch.empty(int(reps), dtype=torch.int32, device=w.device)
    ms = ctypes.c_float()
    _fw.check(_fw.lib().fw_sampler_run(SAMPLERS[method], int(width), _ptr(w), w.numel(), int(reps),
                                       seed & 0xFFFFFFFFFFFFFFFF, _ptr(out), _stream_handle(stream),
                                       ctypes.byref(ms) if timed else None))
    return out, (ms.value if timed else None)
