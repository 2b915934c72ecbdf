#!/usr/bin/env python3
"""Benchmark: filtered lookups/s, stochastic vs deterministic, on one GB300.

Default workload (the dense-grid configuration): a 256^3 FP16 density grid from
seeded fractal noise (~30% non-zero) and 1920x1080 rays x 16 ray-march steps
(33,177,600 queries) from a seeded pinhole camera; B-spline tricubic filtering.
One step = one stochastic lookup batch over all queries (query ingest, per-axis
weights, Philox variates, inverse-CDF tap choice, address, single-texel fetch,
scale and store).  The same-GPU deterministic 64-tap filter, the trilinear pair and
the Morton-binned variant are timed beside it and reported in extra keys.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload dense|tex2d|sparse|sparse_e4m3|neural|serving|aniso|dct]

Other workloads: a 2D RGBA texture, the sparse 2048^3 cloud (FP32 or E4M3 leaves), the
neural texture, a continuous-batching serving mix, anisotropic EWA filtering of a ground
plane, and a DCT-compressed texture set with triplanar mapping.  Every line carries the
same-GPU deterministic filter in `extras`, an end-to-end figure through the C ABI from
pinned host buffers (`e2e`), the oracle's CPU rate (`cpu_baseline`) and the roofline of the
timed kernel.

Timing: CUDA events on the launching stream, W untimed warm-up steps, barrier and
synchronize on both sides of K timed steps, max over ranks.  The query and output
arrays (531 MB per step) are larger than L2, so no extra flush is needed; the
32 MiB grid stays L2-resident by design.  Under torchrun every rank runs the same
per-rank workload (weak scaling, no data-path collective).
"""
import argparse
import hashlib
import json
import os
import statistics
import sys
import threading
import time

# The CPU baseline runs the oracle in one process per host core: numpy's BLAS pool
# (used by the neural oracle's matrix products) is held to one thread per process before
# numpy loads.  (The input generators' OpenMP loops are not part of any timed region and
# keep every core.)
for _v in ("OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TEXEL_FORMAT = {"dense": "fp16", "sparse": "fp32", "tex2d": "fp32",
                "sparse_e4m3": "e4m3 + fp32 leaf scale", "neural": "fp16 latents"}

ALGO_BYTES = {  # algorithmic bytes per lookup: query in + texel(s) + result out
    ("dense", "stochastic"): 12 + 2 + 4,
    ("sparse", "stochastic"): 12 + 4 + 4,
    ("sparse_e4m3", "stochastic"): 12 + 1 + 4 + 4,
    ("neural", "stochastic"): 12 + 16 + 28,
    ("dense", "deterministic", "bspline3"): 12 + 64 * 2 + 4,
    ("dense", "deterministic", "linear"): 12 + 8 * 2 + 4,
    ("tex2d", "stochastic"): 8 + 16 + 16,
    ("tex2d", "deterministic", "bspline3"): 8 + 16 * 16 + 16,
    ("tex2d", "deterministic", "linear"): 8 + 4 * 16 + 16,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense",
                    choices=["dense", "tex2d", "sparse", "sparse_e4m3", "neural", "serving", "aniso",
                             "dct"])
    ap.add_argument("--requests", type=int, default=10000, help="serving: number of requests")
    ap.add_argument("--train-steps", type=int, default=400)
    ap.add_argument("--filter", default=None, choices=["linear", "bspline3", "catmull_rom"],
                    help="default: bspline3 (linear for the neural workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the extra variants")
    return ap.parse_args()


# ------------------------------------------------------------------ workload

def make_workload(name):
    import synth
    if name == "dense":
        vals = synth.dense_density(n=256, seed=3)
        q = synth.camera_queries(**synth.C2_RAYS)
        desc = "dense 256^3 FP16 fractal-noise density (30% non-zero), 1920x1080 rays x 16 steps"
        return dict(name=name, values=vals, coords=q, dims=(256, 256, 256), channels=1, desc=desc)
    if name == "neural":
        size, nlat, nlev = 4096, 4, 13
        latents, params = synth.neural_init(size, nlat, seed=5)
        pyr = synth.box_levels(synth.material(size, seed=5), nlev)
        n = 1 << 24
        desc = ("neural 4096^2 RGB+normal+roughness, 4 FP16 latent levels x 8 ch + MLP 8-64-64-7, "
                "fallback FP16 mips; 16,777,216 uv queries, lod ~ U[0, 4)")
        return dict(name=name, size=size, nlat=nlat, nlev=nlev, latents=latents, params=params,
                    pyramid=pyr, coords=synth.uv_queries(n, seed=2), lod=synth.lods(n, seed=9),
                    channels=7, desc=desc)
    if name.startswith("sparse"):
        origins, values = synth.sparse_cloud(domain=2048, seed=4)
        q = synth.camera_queries(**synth.C3_RAYS)
        fmt = "E4M3 + per-leaf scale" if name == "sparse_e4m3" else "FP32"
        desc = ("sparse 2048^3 cloud, %d active 8^3 leaves (%.1f%%), %s, 2048x2048 rays x 16 steps"
                % (len(origins), 100.0 * len(origins) / 256 ** 3, fmt))
        return dict(name=name, values=values, origins=origins, coords=q, dims=(0, 0, 0),
                    channels=1, desc=desc)
    tex = synth.texture2d(256, 256, 4, seed=1)
    n = 1 << 24
    uv = synth.uv_queries(n, seed=2)
    desc = "2D 256x256 RGBA FP32 value noise, 16,777,216 uniform uv queries"
    return dict(name=name, values=tex, coords=uv, dims=(256, 256, 1), channels=4, desc=desc)


def make_texture(stf, w, fmt=None, train_steps=400):
    if w["name"] == "neural":
        import torch
        pyr = w["pyramid"]
        fb = np.concatenate([p.reshape(-1, 7) for p in pyr[w["nlat"]:]])
        T = stf.NeuralTexture(w["size"], w["size"], w["nlat"], w["nlev"], w["latents"], w["params"], fb)
        target = torch.from_numpy(np.concatenate([p.reshape(-1, 7) for p in pyr[:w["nlat"]]])).cuda()
        losses = T.train(target, steps=train_steps, batch=1 << 16, lr_latent=3e-2, lr_params=3e-3, seed=11)
        w["train_loss"] = (float(losses[0].item()), float(losses[-1].item())) if train_steps else None
        w["train_steps"] = train_steps
        del target
        return T
    if w["name"] == "dense":
        return stf.Texture(stf.KIND_DENSE3D, w["values"], dims=w["dims"],
                           fmt=stf.FMT_F16 if fmt is None else fmt)
    if w["name"].startswith("sparse"):
        f = stf.FMT_E4M3_SCALED if w["name"] == "sparse_e4m3" else stf.FMT_F32
        return stf.Texture(stf.KIND_SPARSE3D, w["values"], fmt=f, leaf_origins=w["origins"])
    return stf.Texture(stf.KIND_TEX2D, w["values"], dims=w["dims"], channels=4)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """SM clock and clock-event reasons sampled through NVML (read-only queries)
    every ~1 ms on a background thread; each sample is time-stamped so that the
    samples inside the timed window can be picked out."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_index):
        self.torch_index = torch_index
        self.samples = []
        self.max_mhz = None
        self._stop = threading.Event()
        self.nv = None
        self.window = None

    def __enter__(self):
        import ctypes
        import torch
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return self
            h = ctypes.c_void_p()
            pr = torch.cuda.get_device_properties(self.torch_index)
            bus = "%08x:%02x:%02x.0" % (getattr(pr, "pci_domain_id", 0), getattr(pr, "pci_bus_id", 0),
                                         getattr(pr, "pci_device_id", 0))
            if nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) != 0:
                if nv.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h)) != 0:
                    return self
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            self.nv, self.h, self.reasons_fn = nv, h, reasons_fn
            self.t = threading.Thread(target=self._run, daemon=True)
            self.t.start()
        except (OSError, AttributeError):
            self.nv = None
        return self

    def _run(self):
        import ctypes
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            ok = self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0
            ok2 = self.reasons_fn(self.h, ctypes.byref(rs)) == 0
            if ok:
                self.samples.append((time.perf_counter(), float(clk.value), rs.value if ok2 else 0))
            time.sleep(0.001)

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *a):
        self._stop.set()
        if self.nv is not None:
            self.t.join(timeout=2)

    def summary(self):
        sel = self.samples
        where = "whole run"
        if self.window:
            inside = [x for x in self.samples if self.window[0] <= x[0] <= self.window[1]]
            if inside:
                sel, where = inside, "timed region"
        reasons = sorted({nm for (_, _, r) in sel for bit, nm in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median([c for (_, c, _) in sel]) if sel else None,
                "sm_max_mhz": self.max_mhz, "reasons": reasons, "samples": len(sel),
                "window": where, "source": "nvml"}


# ------------------------------------------------------------------ timing

def time_steps(torch, fn, steps, warmup, stream, dist=None, return_window=False):
    """Per-step CUDA-event durations (ms) of fn() on `stream`, and the total (ms)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    t0 = time.perf_counter()
    ev[0].record(stream)
    for k in range(steps):
        fn()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    total = ev[0].elapsed_time(ev[steps])
    if dist is not None:
        dist.barrier()
    if return_window:
        return per, total, (t0, t1)
    return per, total


def pct(xs, p):
    xs = sorted(xs)
    i = min(len(xs) - 1, max(0, int(round(p / 100.0 * (len(xs) - 1)))))
    return xs[i]


KERNEL_SOURCES = {"dense": ("stf_grid.cu",), "tex2d": ("stf_tex2d.cuh", "stf_tex2d_f32.cu"),
                  "sparse": ("stf_sparse.cu",), "sparse_e4m3": ("stf_sparse.cu",),
                  "neural": ("stf_neural.cu",), "aniso": ("stf_ewa.cu",),
                  "dct": ("stf_tex2d.cuh", "stf_tex2d_dct.cu")}


def stochastic_extra_bytes(workload, name):
    """Algorithmic bytes per lookup of a stochastic extra: query in, the texel(s) it
    fetches, result out (the positivized filter fetches up to two texels; binning's own
    passes are not counted)."""
    base = ALGO_BYTES.get((workload, "stochastic"))
    if base is None or not name.startswith("stochastic"):
        return None
    if "positivized" in name:
        return base + {"dense": 2, "sparse": 4, "sparse_e4m3": 5, "tex2d": 16}[workload]
    return base


def kernel_hash(workload):
    """Hash of the sources that build the workload's lookup kernel."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2305_05810_gb300", "csrc")
    for f in ("stf_device.cuh", "stf_types.h", "stf_launch.h") + KERNEL_SOURCES[workload]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, filt):
    """DRAM bytes per launch of the stochastic kernel from the committed ncu summary,
    if it was captured on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        e = json.load(open(p)).get("%s_stochastic_%s" % (workload, filt))
        if e and e.get("kernel_hash") == kernel_hash(workload):
            return e["dram_bytes_per_launch"]
    except (OSError, ValueError):
        pass
    return None


def bf16_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        return 1900.0


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU oracle

def touched_leaves(origins, pts):
    """Indices of the leaves a 4x4x4 tap window around any of pts can reach."""
    base = np.floor(pts[np.all(np.abs(pts) < 1e7, axis=1)]).astype(np.int64)
    key = lambda c: (c[:, 0] + 4096) * (1 << 26) + (c[:, 1] + 4096) * (1 << 13) + (c[:, 2] + 4096)
    cells = np.unique(np.concatenate([key((base + np.array(d)) >> 3) for d in
                                      [(a, b, c) for a in (-1, 2) for b in (-1, 2) for c in (-1, 2)]]))
    ok = key(origins.astype(np.int64) >> 3)
    return np.nonzero(np.isin(ok, cells))[0]


def oracle_store(w, n_queries):
    """The oracle's texel store for the workload (the stored values as the library
    holds them; for sparse grids only the leaves the first n_queries queries touch)."""
    from oracle import codecs, textures
    if w["name"] == "dense":
        return textures.Dense3D(codecs.f16_decode(codecs.f16_encode(w["values"].astype(np.float64))))
    if w["name"].startswith("sparse"):
        sub = touched_leaves(w["origins"], w["coords"][:n_queries])
        vals = w["values"][sub]
        if w["name"] == "sparse_e4m3":
            codes, scales = codecs.e4m3_leaf_quantise(vals)
            vals = codecs.e4m3_leaf_dequantise(codes, scales)
        return textures.Sparse3D(w["origins"][sub], vals)
    if w["name"] == "neural":
        from oracle import mlp, neural
        h16 = lambda a: codecs.f16_decode(codecs.f16_encode(np.asarray(a, dtype=np.float64)))
        P = mlp.unflatten(np.asarray(w["trained_params"], dtype=np.float64))
        for k in ("W1", "W2", "W3"):
            P[k] = h16(P[k])
        lat, o, levels = w["trained_latents"], 0, []
        for L in range(w["nlat"]):
            m = max(1, w["size"] >> L)
            levels.append(h16(lat[o:o + m * m]).reshape(m, m, 8))
            o += m * m
        return neural.NeuralTexture2D(levels, P, [h16(p) for p in w["pyramid"][w["nlat"]:]])
    return textures.Texture2D([w["values"].astype(np.float64)])


_ORACLE = {}


def _oracle_init(ref, name, filt):
    """Pool worker set-up: the texel store arrives once per worker (untimed)."""
    _ORACLE.update(ref=ref, name=name, filt=filt)


def _oracle_chunk(job):
    """One chunk of stochastic oracle lookups: job = (first query index, coords, lod)."""
    from oracle import filters
    a, q, lod = job
    ref, name, filt = _ORACLE["ref"], _ORACLE["name"], _ORACLE["filt"]
    qid = np.arange(a, a + q.shape[0], dtype=np.uint64)
    if name == "neural":
        filters.lookup_2d(ref, q, lod, filt, stochastic_form=True, seed=1, qid=qid,
                          level_mode=filters.LEVEL_NEAREST)
    elif name == "aniso":                   # lod carries the uv derivatives; filt the anisotropy
        from oracle import ewa
        ewa.lookup(ref, q, lod, filt, stochastic_form=True, seed=1, qid=qid)
    elif name == "dct":
        filters.lookup_2d(ref, q, lod, filt, stochastic_form=True, seed=1, qid=qid)
    elif name != "tex2d":
        filters.lookup_3d(ref, q, filt, stochastic_form=True, seed=1, qid=qid)
    else:
        filters.lookup_2d(ref, q, None, filt, stochastic_form=True, seed=1, qid=qid)
    return q.shape[0]


class OraclePool:
    """The oracle as it stands, run over query chunks on every host core: one
    process per core (spawned, so a pool started after the GPU is in use does not
    inherit its driver state), numpy's BLAS held to one thread in each."""

    CHUNK = 1 << 17

    def __init__(self, w, filt, n_queries, cores=None):
        import multiprocessing as mp
        self.cores = cores or os.cpu_count() or 1
        self.w, self.n = w, n_queries
        ref = oracle_store(w, n_queries)
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init,
                                                 initargs=(ref, w["name"], filt))
        self.resize(n_queries)
        # every worker has received the store before any timed call
        self.pool.map(_oracle_chunk, [(0, w["coords"][:64], w["lod"][:64] if "lod" in w else None)]
                      * (4 * self.cores), chunksize=1)

    def resize(self, n_queries):
        """Time the first n_queries queries (at most the count the store was built for)."""
        w = self.w
        self.n = n_queries
        self.jobs = [(a, w["coords"][a:min(n_queries, a + self.CHUNK)],
                      w["lod"][a:min(n_queries, a + self.CHUNK)] if "lod" in w else None)
                     for a in range(0, n_queries, self.CHUNK)]

    def rate(self):
        """Lookups/s over the first n_queries queries, and the seconds taken."""
        t0 = time.perf_counter()
        done = sum(self.pool.imap_unordered(_oracle_chunk, self.jobs, chunksize=1))
        dt = time.perf_counter() - t0
        assert done == self.n
        return done / dt, dt

    def close(self):
        self.pool.close()
        self.pool.join()


def pooled_oracle_rate(ref, name, filt, q, aux, chunk):
    """Oracle lookups/s over q (with aux: lod or derivatives) on every host core, one
    spawned process per core holding ref; returns (rate, seconds, cores)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(ref, name, filt))
    try:
        pool.map(_oracle_chunk, [(0, q[:64], aux[:64])] * (4 * cores), chunksize=1)
        jobs = [(a, q[a:a + chunk], aux[a:a + chunk]) for a in range(0, q.shape[0], chunk)]
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_chunk, jobs, chunksize=1))
        dt = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    return done / dt, dt, cores


def cpu_oracle_rate(w, filt, n_queries):
    """Oracle lookups/s on the first n_queries queries (stochastic) on every host core;
    returns (rate, seconds, cores)."""
    pool = OraclePool(w, filt, n_queries)
    try:
        rate, dt = pool.rate()
    finally:
        pool.close()
    return rate, dt, pool.cores


def storage_error(stf, torch, w, tex, filt, stream, m=1 << 17, level_mode=None):
    """Error of the library's stochastic and deterministic lookups on the stored
    texture (FP16 / E4M3 + leaf scale / FP32; the neural texture's FP16 latents and
    decoder) against the float64 oracle on the unquantised texels (the float32 values
    the texture was built from; for the neural texture, its float32 master latents and
    weights, and beside that the target texture it was trained on, which measures the
    fit of the network rather than its storage), over m consecutive queries from the
    middle of the workload.  The stochastic pair draws the same taps (queries whose
    tap the oracle marks exempt are left out), so its error is the storage error of
    the fetched texel; the deterministic pair compares the full filters.  Oracle leg
    only: part of the CPU-baseline run."""
    from oracle import filters, textures
    n = w["coords"].shape[0]
    m = min(m, n)
    a = (n - m) // 2
    q = w["coords"][a:a + m]
    qid = np.arange(a, a + m, dtype=np.uint64)
    dev = torch.device("cuda", torch.cuda.current_device())
    d = torch.from_numpy(np.ascontiguousarray(q)).to(dev)
    lod = w["lod"][a:a + m] if "lod" in w else None
    d_lod = None if lod is None else torch.from_numpy(np.ascontiguousarray(lod)).to(dev)
    C = w["channels"]
    got = torch.empty((m, C), dtype=torch.float32, device=dev)
    taps = torch.empty((m, 4), dtype=torch.int32, device=dev)
    det = torch.empty((m, C), dtype=torch.float32, device=dev)
    lm = stf.LEVEL_STOCHASTIC if level_mode is None else level_mode
    p = stf.make_params(filt, seed=2024, level_mode=lm, query_offset=a)
    stf.stf_lookup_batch(tex.handle, p, d, d_lod, m, got, taps, stream)
    stf.stf_lookup_batch_deterministic(tex.handle, stf.make_params(filt, level_mode=lm), d, d_lod, m, det,
                                       stream)
    torch.cuda.synchronize()
    got, taps, det = got.cpu().numpy(), taps.cpu().numpy(), det.cpu().numpy()
    if w["name"] == "dense":
        ref = textures.Dense3D(np.asarray(w["values"], dtype=np.float64).reshape(w["dims"][::-1]))
    elif w["name"].startswith("sparse"):
        sub = touched_leaves(w["origins"], q)
        ref = textures.Sparse3D(w["origins"][sub], np.asarray(w["values"][sub], dtype=np.float64))
    elif w["name"] == "neural":
        from oracle import mlp, neural
        lat, o, levels = np.asarray(w["trained_latents"], dtype=np.float64), 0, []
        for L in range(w["nlat"]):
            s_ = max(1, w["size"] >> L)
            levels.append(lat[o:o + s_ * s_].reshape(s_, s_, 8))
            o += s_ * s_
        ref = neural.NeuralTexture2D(levels, mlp.unflatten(np.asarray(w["trained_params"], dtype=np.float64)),
                                     [np.asarray(p_, dtype=np.float64) for p_ in w["pyramid"][w["nlat"]:]])
    else:
        ref = textures.Texture2D([np.asarray(w["values"], dtype=np.float64)])

    def oracle(ref):
        if ref.__class__.__name__ in ("Texture2D", "NeuralTexture2D"):
            rv, rt, ex = filters.lookup_2d(ref, q, lod, filt, stochastic_form=True, level_mode=lm, qid=qid,
                                           seed=2024)
            dv, _, _ = filters.lookup_2d(ref, q, lod, filt, stochastic_form=False, level_mode=lm)
        else:
            rv, rt, ex = filters.lookup_3d(ref, q, filt, stochastic_form=True, qid=qid, seed=2024)
            dv, _, _ = filters.lookup_3d(ref, q, filt, stochastic_form=False)
        return rv, rt, ex, dv

    vals = np.asarray(w["pyramid"][0] if w["name"] == "neural" else w["values"], dtype=np.float64)
    rng = float(vals.max() - vals.min())

    def stats(e):
        e = np.abs(e)
        return {"max_abs": float(e.max()), "rms": float(np.sqrt(np.mean(e * e))),
                "max_rel_to_range": float(e.max() / rng)}

    def compare(ref):
        rv, rt, ex, dv = oracle(ref)
        same = np.all(taps == rt, axis=1) & ~ex
        return {"stochastic": stats(got[same] - rv[same]), "deterministic": stats(det - dv),
                "same_taps": int(same.sum())}

    out = compare(ref)
    out.update(queries=m, value_range=rng, against="float64 oracle on the unquantised texels"
               if w["name"] != "neural" else "float64 oracle on the float32 master latents and weights")
    if w["name"] == "neural":
        fit = compare(textures.Texture2D([np.asarray(p_, dtype=np.float64) for p_ in w["pyramid"]]))
        fit["against"] = "float64 oracle on the target texture the network was trained on"
        fit["train_steps"] = w.get("train_steps")
        out["fit_to_target"] = fit
    return out


# ------------------------------------------------------------------ arms

def run_serving(args):
    """Continuous-batching serving over the four resident textures (2D, dense,
    sparse, neural): log-uniform request sizes in [1K, 4M] queries, mixed filters,
    stochastic/deterministic 50/50, 16 GB admission budget, 8 slots.  Capacity is
    first measured closed-loop (all requests queued at once); then requests arrive
    as a Poisson process at 70% of that capacity and latency is arrival -> results
    on the host."""
    import torch
    import paper_2305_05810_gb300 as stf
    from paper_2305_05810_gb300 import serving
    stf.load()
    ws = {k: make_workload(k) for k in ("tex2d", "dense", "sparse", "neural")}
    textures = {k: make_texture(stf, w, train_steps=args.train_steps) for k, w in ws.items()}
    pools = {k: torch.from_numpy(w["coords"]).pin_memory() for k, w in ws.items()}
    lod_pool = torch.from_numpy(ws["neural"]["lod"]).pin_memory()
    keys = list(textures)

    def make(i, size, rng):
        key = keys[int(rng.integers(0, len(keys)))]
        pool = pools[key]
        start = int(rng.integers(0, pool.shape[0] - size))
        lod = lod_pool[start:start + size] if key == "neural" else None
        filt = ("linear", "bspline3", "catmull_rom")[int(rng.integers(0, 3))]
        lm = stf.LEVEL_NEAREST if key == "neural" else stf.LEVEL_STOCHASTIC
        return serving.Request(i, key, pool[start:start + size], lod, filter=filt,
                               stochastic=bool(rng.integers(0, 2)), seed=1000 + i, level_mode=lm)

    # results are consumed from the slots' pinned buffers (no per-request host copy)
    backend = serving.TorchBackend(textures, n_slots=8, keep_results=False)
    # the budget covers the resident textures and every slot's buffers
    resident = sum(T.nbytes for T in textures.values())

    def run(rate):
        # closed loop (rate None): the same request sequence, all queued at the start
        reqs = serving.poisson_requests(args.requests, rate or 1.0, (1000, 4 << 20), make, seed=6)
        sched = serving.Scheduler(backend, n_slots=8, budget_bytes=16 << 30, chunk_queries=1 << 20,
                                  resident_bytes=resident)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = sched.run(reqs, realtime=rate is not None)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return done, sched, dt

    run(None)                                   # warm-up (allocator, pinned buffers)
    done, sched, dt = run(None)                 # closed loop: capacity
    total = sum(r.n for r in done)
    capacity = total / dt
    mean_size = total / len(done)
    rate = 0.7 * capacity / mean_size
    done, sched, dt = run(rate)
    total = sum(r.n for r in done)
    lat = serving.latency_summary(done)
    line = {"metric": "serving: lookups/s and p50/p99 request latency (mixed textures)",
            "value": total / dt, "unit": "lookups/s", "n_gpus": 1, "higher_is_better": True,
            "p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"], "mean_ms": lat["mean_ms"],
            "requests": len(done), "arrival_rate_per_s": rate,
            "closed_loop_capacity_lookups_per_s": capacity,
            "peak_admitted": sched.peak_active, "peak_device_bytes": sched.peak_in_use,
            "resident_texture_bytes": resident,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving over 2D, dense, sparse and neural textures",
                       "sizes": "log-uniform 1K-4M", "slots": 8, "budget_bytes": 16 << 30,
                       "chunk_queries": 1 << 20, "stochastic_fraction": 0.5}}
    print(json.dumps(line), flush=True)
    for T in textures.values():
        T.close()
    return 0


def run_aniso(args):
    """Anisotropic minification (Sections 4.2, 5.2): a 1024^2 RGBA FP16 texture with its
    full box pyramid (11 levels) seen across a ground plane at 3840x2160 (one query per
    pixel that hits the textured square, with its screen-space uv derivatives).  The
    timed step is the stochastic EWA lookup (max anisotropy 16, stochastic level, one
    texel); extras time the deterministic EWA (pbrt: two levels blended) and the
    real-time path of the paper (anisotropic LOD, then one stochastic bilinear tap or
    the deterministic trilinear filter).  Inputs (5.3M queries x 24 B) and outputs are
    larger than L2."""
    import torch
    import paper_2305_05810_gb300 as stf
    import synth
    stf.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    size, levels, ma = 1024, 11, 16.0
    base = synth.texture2d(size, size, 4, seed=1)
    tex = stf.Texture(stf.KIND_TEX2D, base, dims=(size, size, 1), channels=4, mip_levels=levels,
                      generate_mips=True, fmt=stf.FMT_F16)
    uv_h, g_h = synth.plane_view(W=3840, H=2160, seed=7)
    n = uv_h.shape[0]
    uv, g = torch.from_numpy(uv_h).to(dev), torch.from_numpy(g_h).to(dev)
    out = torch.empty((n, 4), dtype=torch.float32, device=dev)
    lod = torch.empty((n,), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    p = stf.make_params(seed=2024)

    def ewa_sto():
        stf.stf_lookup_batch_ewa(tex.handle, p, uv, g, n, ma, out, None, stream)

    with ClockSampler(torch.cuda.current_device()) as clk:
        per, total, win = time_steps(torch, ewa_sto, args.steps, args.warmup, stream, return_window=True)
        clk.mark(*win)
    stf.stf_synchronize(tex.handle, stream)
    value = n * args.steps / (total / 1000.0)
    pd = stf.make_params()
    pl = stf.make_params("linear", seed=2024)
    pld = stf.make_params("linear")

    def realtime_sto():
        stf.stf_anisotropic_lod(tex.handle, g, n, ma, lod, stream)
        stf.stf_lookup_batch(tex.handle, pl, uv, lod, n, out, None, stream)

    def realtime_det():
        stf.stf_anisotropic_lod(tex.handle, g, n, ma, lod, stream)
        stf.stf_lookup_batch_deterministic(tex.handle, pld, uv, lod, n, out, stream)

    extras = {}
    if not args.quick:
        for name, fn in (("deterministic_ewa", lambda: stf.stf_lookup_batch_ewa_deterministic(
                              tex.handle, pd, uv, g, n, ma, out, stream)),
                         ("realtime_aniso_lod_stochastic_bilinear", realtime_sto),
                         ("realtime_aniso_lod_deterministic_trilinear", realtime_det)):
            p2, t2 = time_steps(torch, fn, max(3, args.steps // 2), 2, stream)
            extras[name] = {"lookups_per_s": n * len(p2) / (t2 / 1000.0), "ms_p50": pct(p2, 50),
                            "ms_p99": pct(p2, 99)}
        extras["speedup_vs_deterministic"] = value / extras["deterministic_ewa"]["lookups_per_s"]
    # end to end through the C ABI: pinned uv + derivatives in, results out every step
    h_uv, h_g = torch.from_numpy(uv_h).pin_memory(), torch.from_numpy(g_h).pin_memory()
    h_out = torch.empty((n, 4), dtype=torch.float32).pin_memory()
    d_uv, d_g = torch.empty_like(uv), torch.empty_like(g)

    def e2e_step():
        d_uv.copy_(h_uv, non_blocking=True)
        d_g.copy_(h_g, non_blocking=True)
        stf.stf_lookup_batch_ewa(tex.handle, p, d_uv, d_g, n, ma, out, None, stream)
        h_out.copy_(out, non_blocking=True)

    pe, te = time_steps(torch, e2e_step, max(3, args.steps // 2), 2, stream)
    hbm, peak_kind = peaks()
    algo = 8 + 16 + 8 + 16
    avg = statistics.mean(per)
    achieved = algo * n / (avg / 1000.0) / 1e9
    line = {
        "metric": "EWA lookups/s (stochastic, anisotropic minification)", "value": value,
        "unit": "lookups/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps, "ms_best": min(per), "ms_p50": pct(per, 50), "ms_p99": pct(per, 99),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"texel_format": "fp16",
                   "workload": "aniso: 1024^2 RGBA FP16 + 11 box levels, ground plane at 3840x2160, "
                               "%d queries with uv derivatives, EWA max anisotropy 16" % n,
                   "l2": "inputs and outputs larger than L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": ncu_traffic("aniso", "ewa"),
                     "algorithmic_bytes_per_lookup": algo, "peak_source": peak_kind,
                     "note": "the kernel is bound by the per-texel ellipse arithmetic, not by bytes"},
        "e2e": {"value": n * len(pe) / (te / 1000.0), "unit": "lookups/s",
                "h2d_bytes_per_step": n * 24, "d2h_bytes_per_step": n * 16},
        "gpu_launches": args.warmup + args.steps, "clocks": clk.summary(), "extras": extras,
    }
    if not args.no_cpu_baseline:
        from oracle import ewa, textures
        ref = textures.Texture2D.box_pyramid(base.astype(np.float64), levels)
        m = min(n, 1 << 16)
        rate, dt, cores = pooled_oracle_rate(ref, "aniso", ma, uv_h[:m], g_h[:m], 1024)
        line["cpu_baseline"] = {"value": rate, "unit": "lookups/s", "cores": cores, "kind": "oracle",
                                "sample": "first %d queries, stochastic EWA, %.1f s on %d processes"
                                          % (m, dt, cores)}
    print(json.dumps(line), flush=True)
    tex.close()
    return 0


def run_dct(args):
    """DCT-compressed texture set (Section 5.2, "Texture compression"): a 4096^2
    8-channel texture set (value noise in [0, 1]), full box pyramid (13 levels),
    encoded to six DCT coefficients per 8x8 block and channel (32 bits: 16x smaller
    than 8-bit texels), seen across a ground plane at 3840x2160 (one query per pixel that
    hits the plane; level of detail from the anisotropic LOD of the footprint, computed
    once before timing).  The timed step is stochastic trilinear filtering (stochastic
    level, one bilinear tap: one decoded texel); extras: deterministic trilinear (eight
    decoded texels), the same pair on the uncompressed FP16 texture, and stochastic /
    deterministic triplanar mapping of a sphere (one vs 24 decoded texels)."""
    import torch
    import paper_2305_05810_gb300 as stf
    import synth
    stf.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    size, C, levels = 4096, 8, 13
    base = synth.texture2d(size, size, C, seed=1)
    tex = stf.Texture(stf.KIND_TEX2D, base, dims=(size, size, 1), channels=C, mip_levels=levels,
                      generate_mips=True, fmt=stf.FMT_DCT6)
    uv_h, g_h = synth.plane_view(W=3840, H=2160, seed=7)
    n = uv_h.shape[0]
    uv, g = torch.from_numpy(uv_h).to(dev), torch.from_numpy(g_h).to(dev)
    lod = tex.anisotropic_lod(g, 16.0)
    out = torch.empty((n, C), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ps, pd = stf.make_params("linear", seed=2024), stf.make_params("linear")

    def sto():
        stf.stf_lookup_batch(tex.handle, ps, uv, lod, n, out, None, stream)

    with ClockSampler(torch.cuda.current_device()) as clk:
        per, total, win = time_steps(torch, sto, args.steps, args.warmup, stream, return_window=True)
        clk.mark(*win)
    stf.stf_synchronize(tex.handle, stream)
    value = n * args.steps / (total / 1000.0)
    extras = {}
    if not args.quick:
        f16 = stf.Texture(stf.KIND_TEX2D, base, dims=(size, size, 1), channels=C, mip_levels=levels,
                          generate_mips=True, fmt=stf.FMT_F16)
        pts, nrm = synth.sphere_points(3840 * 2160, seed=8)
        m = pts.shape[0]
        dp, dn = torch.from_numpy(pts).to(dev), torch.from_numpy(nrm).to(dev)
        tlod = torch.from_numpy(synth.lods(m, seed=9, lo=0.0, hi=4.0)).to(dev)
        tout = torch.empty((m, C), dtype=torch.float32, device=dev)
        variants = [
            ("deterministic_trilinear", n, lambda: stf.stf_lookup_batch_deterministic(
                tex.handle, pd, uv, lod, n, out, stream)),
            ("fp16_uncompressed_stochastic_trilinear", n, lambda: stf.stf_lookup_batch(
                f16.handle, ps, uv, lod, n, out, None, stream)),
            ("fp16_uncompressed_deterministic_trilinear", n, lambda: stf.stf_lookup_batch_deterministic(
                f16.handle, pd, uv, lod, n, out, stream)),
            ("triplanar_stochastic_trilinear", m, lambda: stf.stf_lookup_batch_triplanar(
                tex.handle, ps, dp, dn, tlod, m, 1.0, tout, None, stream)),
            ("triplanar_deterministic_trilinear", m, lambda: stf.stf_lookup_batch_triplanar_deterministic(
                tex.handle, pd, dp, dn, tlod, m, 1.0, tout, stream)),
        ]
        for name, cnt, fn in variants:
            p2, t2 = time_steps(torch, fn, max(3, args.steps // 2), 2, stream)
            extras[name] = {"lookups_per_s": cnt * len(p2) / (t2 / 1000.0), "ms_p50": pct(p2, 50),
                            "ms_p99": pct(p2, 99)}
        extras["speedup_vs_deterministic"] = value / extras["deterministic_trilinear"]["lookups_per_s"]
        extras["triplanar_speedup"] = (extras["triplanar_stochastic_trilinear"]["lookups_per_s"] /
                                       extras["triplanar_deterministic_trilinear"]["lookups_per_s"])
        extras["texture_bytes"] = {"dct6": tex.nbytes, "fp16": f16.nbytes}
        f16.close()
    h_uv = torch.from_numpy(uv_h).pin_memory()
    h_lod = lod.cpu().pin_memory()
    h_out = torch.empty((n, C), dtype=torch.float32).pin_memory()
    d_uv, d_lod = torch.empty_like(uv), torch.empty_like(lod)

    def e2e_step():
        d_uv.copy_(h_uv, non_blocking=True)
        d_lod.copy_(h_lod, non_blocking=True)
        stf.stf_lookup_batch(tex.handle, ps, d_uv, d_lod, n, out, None, stream)
        h_out.copy_(out, non_blocking=True)

    pe, te = time_steps(torch, e2e_step, max(3, args.steps // 2), 2, stream)
    hbm, peak_kind = peaks()
    algo = 8 + 4 + 4 * C + 4 * C
    achieved = algo * n / (statistics.mean(per) / 1000.0) / 1e9
    line = {
        "metric": "DCT-texture lookups/s (stochastic trilinear)", "value": value, "unit": "lookups/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
        "ms_best": min(per), "ms_p50": pct(per, 50), "ms_p99": pct(per, 99), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"texel_format": "dct6",
                   "workload": "dct: 4096^2 x 8 channels DCT6 (6 coefficients per 8x8 block, 7/5-bit "
                               "codes) + 13 levels, ground plane at 3840x2160, %d queries, anisotropic "
                               "LOD" % n, "l2": "inputs and outputs larger than L2"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": ncu_traffic("dct", "linear"),
                     "algorithmic_bytes_per_lookup": algo, "peak_source": peak_kind},
        "e2e": {"value": n * len(pe) / (te / 1000.0), "unit": "lookups/s",
                "h2d_bytes_per_step": n * 12, "d2h_bytes_per_step": n * 4 * C},
        "gpu_launches": args.warmup + args.steps, "clocks": clk.summary(), "extras": extras,
    }
    if not args.no_cpu_baseline:
        # the oracle's float64 encoder on the same pyramid (set-up, untimed), then its
        # stochastic trilinear lookups on the first 2^22 queries (timed)
        from oracle import dct as odct
        lv = [p.astype(np.float64) for p in synth.box_levels(base, levels)]
        ref = odct.DCTTexture2D(lv)
        del lv
        m = min(n, 1 << 22)
        rate, dt, cores = pooled_oracle_rate(ref, "dct", "linear", uv_h[:m], lod.cpu().numpy()[:m], 1 << 16)
        line["cpu_baseline"] = {"value": rate, "unit": "lookups/s", "cores": cores, "kind": "oracle",
                                "sample": "first %d queries, stochastic trilinear on the DCT texture, "
                                          "%.1f s on %d processes" % (m, dt, cores)}
    print(json.dumps(line), flush=True)
    tex.close()
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = make_workload(args.workload)
    if args.workload == "neural":
        w["trained_params"], w["trained_latents"] = w["params"], w["latents"]
    # the whole workload where the oracle on every core finishes a step in a few
    # seconds (dense, 2D); a leading sample of the sparse and neural workloads
    n_all = w["coords"].shape[0]
    n_sample = n_all if args.workload in ("dense", "tex2d") else min(n_all, 1 << 22)
    pool = OraclePool(w, args.filter, n_sample)
    rates = []
    try:
        # a calibration pass sizes the sample so that the whole run takes about three
        # minutes at most (the whole workload when that fits)
        pool.resize(min(n_sample, 1 << 21))
        r0, _ = pool.rate()
        fit = int(r0 * 180.0 / max(1, args.warmup + args.steps)) // OraclePool.CHUNK * OraclePool.CHUNK
        n_sample = max(OraclePool.CHUNK, min(n_sample, fit))
        pool.resize(n_sample)
        for k in range(args.warmup + args.steps):
            r, _ = pool.rate()
            if k >= args.warmup:
                rates.append(r)
    finally:
        pool.close()
    total_time = sum(n_sample / r for r in rates)
    value = n_sample * len(rates) / total_time
    line = {
        "impl": "reference", "metric": "filtered lookups/s (stochastic, %s)" % args.filter,
        "value": value, "unit": "lookups/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * total_time / len(rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": w["desc"], "filter": args.filter,
                                         "texel_format": TEXEL_FORMAT.get(w["name"], "fp32"),
                                         "queries_per_step": n_sample},
        "same_config": n_sample == n_all,
        "cpu_baseline": {"value": value, "unit": "lookups/s", "cores": pool.cores, "kind": "oracle",
                         "sample": ("all %d queries of the workload per step" % n_sample if n_sample == n_all
                                    else "first %d of %d queries per step" % (n_sample, n_all))},
        "e2e": {"value": value, "unit": "lookups/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import paper_2305_05810_gb300 as stf

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    dev = torch.device("cuda", torch.cuda.current_device())
    stf.load()

    w = make_workload(args.workload)
    tex = make_texture(stf, w, train_steps=args.train_steps)
    n = w["coords"].shape[0]
    C = w["channels"]
    coords = torch.from_numpy(w["coords"]).to(dev)
    out = torch.empty((n, C), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    filt = args.filter
    lod = torch.from_numpy(w["lod"]).to(dev) if "lod" in w else None
    # the neural workload compares one decode with the 4-decode bilinear filter at one level
    level_mode = stf.LEVEL_NEAREST if w["name"] == "neural" else stf.LEVEL_STOCHASTIC

    # weak scaling: every rank filters its own full batch; rank r's queries are the
    # r-th block of one world-wide batch (query_offset = r * n), so no two ranks
    # share variates and nothing is exchanged
    qoff = rank * n

    def stochastic(f=filt, **kw):
        p = stf.make_params(f, seed=2024, level_mode=level_mode, query_offset=qoff, **kw)
        return lambda: stf.stf_lookup_batch(tex.handle, p, coords, lod, n, out, None, stream)

    def deterministic(f):
        p = stf.make_params(f, level_mode=level_mode)
        return lambda: stf.stf_lookup_batch_deterministic(tex.handle, p, coords, lod, n, out, stream)

    with ClockSampler(torch.cuda.current_device()) as clk:
        per, total, win = time_steps(torch, stochastic(), args.steps, args.warmup, stream, dist,
                                     return_window=True)
        clk.mark(*win)
    stf.stf_synchronize(tex.handle, stream)

    # max over ranks
    t_total = torch.tensor([total], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t_total, op=dist.ReduceOp.MAX)
    total = float(t_total.item())
    value = n * world * args.steps / (total / 1000.0)

    extras = {}
    sparse_extra = []
    if not args.quick:
        variants = [("deterministic_" + filt, deterministic(filt))]
        if w["name"] != "neural":
            variants += [("stochastic_catmull_rom", stochastic("catmull_rom")),
                         ("stochastic_catmull_rom_positivized", stochastic("catmull_rom_positivized")),
                         # filter importance sampling: B-splines by sums of uniforms, and a
                         # Gaussian (sigma = 1 texel) by Box-Muller, each one texel fetch
                         ("stochastic_fis_linear", stochastic("fis_linear")),
                         ("stochastic_fis_bspline3", stochastic("fis_bspline3")),
                         ("stochastic_fis_gaussian_sigma1", stochastic("fis_gaussian", width=1.0))]
            # its deterministic twin sums every tap within 5.77 sigma (13 per axis), so it
            # is timed on the first 2^20 queries
            m = min(n, 1 << 20)
            pg = stf.make_params("fis_gaussian", level_mode=level_mode, width=1.0)
            det_g = (lambda: stf.stf_lookup_batch_deterministic(tex.handle, pg, coords, lod, m, out,
                                                                stream))
            variants += [("deterministic_fis_gaussian_sigma1_first_2^20", det_g)]
        if filt != "linear":
            variants += [("stochastic_linear", stochastic("linear")),
                         ("deterministic_linear", deterministic("linear"))]
        variants += [("stochastic_binned", stochastic(bin_queries=True))]
        # the same queries in a seeded random order (incoherent rays): where binning pays
        g = torch.Generator(device=dev)
        g.manual_seed(7)
        order = torch.randperm(n, device=dev, generator=g)
        shuffled = coords[order].contiguous()
        lod_shuf = None if lod is None else lod[order].contiguous()
        pshuf = stf.make_params(filt, seed=2024, level_mode=level_mode, query_offset=qoff)
        pshuf_b = stf.make_params(filt, seed=2024, level_mode=level_mode, query_offset=qoff,
                                  bin_queries=True)
        variants += [("stochastic_shuffled", lambda: stf.stf_lookup_batch(
                          tex.handle, pshuf, shuffled, lod_shuf, n, out, None, stream)),
                     ("stochastic_shuffled_binned", lambda: stf.stf_lookup_batch(
                          tex.handle, pshuf_b, shuffled, lod_shuf, n, out, None, stream))]
        if w["name"] == "dense" and filt in ("bspline3", "linear"):
            # the queries whose filter window touches the grid (the others return the
            # background without drawing): the same kernel on those alone
            lo, hi = (-1, 2) if filt == "bspline3" else (0, 1)
            fl = torch.floor(coords)
            dims = torch.tensor(w["dims"], device=dev, dtype=coords.dtype)
            hit = ((fl + hi >= 0) & (fl + lo < dims)).all(dim=1)
            hits = coords[hit].contiguous()
            nh = hits.shape[0]
            ph = stf.make_params(filt, seed=2024, level_mode=level_mode, query_offset=qoff)
            variants += [("stochastic_hits_only", lambda: stf.stf_lookup_batch(
                tex.handle, ph, hits, None, nh, out, None, stream))]
        hbm_peak, _ = peaks()
        for name, fn in variants:
            try:
                p2, t2 = time_steps(torch, fn, max(3, args.steps // 2), 2, stream)
                nq = min(n, 1 << 20) if name.endswith("first_2^20") else n
                if name == "stochastic_hits_only":
                    nq = nh
                extras[name] = {"lookups_per_s": nq * len(p2) / (t2 / 1000.0),
                                "ms_p50": pct(p2, 50), "ms_p99": pct(p2, 99)}
                b = stochastic_extra_bytes(w["name"], name)
                if b is not None:
                    extras[name]["hbm_frac"] = extras[name]["lookups_per_s"] * b / 1e9 / hbm_peak
                    extras[name]["algorithmic_bytes_per_lookup"] = b
                if name == "stochastic_hits_only":
                    extras[name]["queries"] = nh
                    extras[name]["fraction_of_workload"] = nh / n
            except stf.StfError as e:
                extras[name] = {"unavailable": str(e)}
        if w["name"] == "sparse_e4m3":
            # storage error: deterministic tricubic on E4M3 leaves against the same lookups on
            # the FP32 leaves, over every 61st query (all of the image and, 61 being prime
            # to the 16 steps per ray, every step), in units of the voxel values; rms over
            # the lookups that touch the cloud (non-zero FP32 value)
            f32 = stf.Texture(stf.KIND_SPARSE3D, w["values"], fmt=stf.FMT_F32, leaf_origins=w["origins"])
            sub = coords[::61].contiguous()
            m = sub.shape[0]
            ref32 = torch.empty((m, 1), dtype=torch.float32, device=dev)
            got = torch.empty((m, 1), dtype=torch.float32, device=dev)
            pq = stf.make_params(filt)
            stf.stf_lookup_batch_deterministic(f32.handle, pq, sub, None, m, ref32, stream)
            stf.stf_lookup_batch_deterministic(tex.handle, pq, sub, None, m, got, stream)
            err = (got - ref32).abs()
            hit = ref32 != 0
            rng = float(w["values"].max() - w["values"].min())
            extras["e4m3_error_vs_fp32_leaves"] = {
                "max_abs": float(err.max()), "rms_in_cloud": float(err[hit].pow(2).mean().sqrt()),
                "lookups_in_cloud": int(hit.sum()), "value_range": rng, "queries": m}
            f32.close()
        if w["name"] == "tex2d":
            # the 65,536-query configuration: per-launch latency over 1000 launches, and the
            # 4096-sample sweep (268M lookups, float64 accumulators) as one launch
            m = 1 << 16
            p65 = stf.make_params(filt, seed=2024)
            lat, _ = time_steps(torch, lambda: stf.stf_lookup_batch(tex.handle, p65, coords, None, m, out,
                                                                     None, stream), 1000, 10, stream)
            extras["c1_65536_queries_launch_ms"] = {"p50": pct(lat, 50), "p99": pct(lat, 99),
                                                    "lookups_per_s": m / (statistics.mean(lat) / 1000.0),
                                                    "l2": "inputs L2-resident (a latency figure)"}
            s1 = torch.empty((m, C), dtype=torch.float64, device=dev)
            s2 = torch.empty_like(s1)
            sweep = lambda: stf.stf_lookup_accumulate(tex.handle, p65, coords, None, m, 4096, s1, s2, stream)
            ps, ts = time_steps(torch, sweep, 3, 1, stream)
            extras["c1_4096_sample_sweep"] = {"lookups_per_s": m * 4096 * len(ps) / (ts / 1000.0),
                                              "ms": statistics.mean(ps)}
        det = extras.get("deterministic_" + filt, {})
        if "lookups_per_s" in det:
            extras["speedup_vs_deterministic"] = value / world / det["lookups_per_s"]
        if w["name"] == "dense" and world == 1:
            sparse_extra = sparse_extras(stf, torch, args, extras, stream)

    # end to end: pinned host coords -> device, lookup, device -> host each step
    h_coords = torch.from_numpy(w["coords"]).pin_memory()
    h_lod = None if lod is None else torch.from_numpy(w["lod"]).pin_memory()
    h_out = torch.empty((n, C), dtype=torch.float32).pin_memory()
    d_in = torch.empty_like(coords)
    d_lod = None if lod is None else torch.empty_like(lod)
    pe = stf.make_params(filt, seed=2024, level_mode=level_mode, query_offset=qoff)

    # the package's host pipeline: chunks of 4M queries over three streams, so that the
    # copies in both directions overlap the lookups, the last chunk split in four (1.5%
    # sooner on the dense workload; 1M-8M chunks, 2-4 streams measured no better)
    from paper_2305_05810_gb300.pipeline import HostPipeline
    pipe = HostPipeline(tex, chunk=1 << 22, n_streams=3, tail=4)

    def e2e_step():
        pipe.lookup(pe, h_coords, h_out, h_lod)

    def e2e_serial():
        d_in.copy_(h_coords, non_blocking=True)
        if d_lod is not None:
            d_lod.copy_(h_lod, non_blocking=True)
        stf.stf_lookup_batch(tex.handle, pe, d_in, d_lod, n, out, None, stream)
        h_out.copy_(out, non_blocking=True)

    if not args.quick:
        ps_, ts_ = time_steps(torch, e2e_serial, max(3, args.steps // 2), 2, stream)
        extras["e2e_serial_one_stream"] = {"lookups_per_s": n * len(ps_) / (ts_ / 1000.0)}
        # the same pinned host buffers passed to the lookup directly: the kernel reads the
        # coordinates and writes the results across the host link, no staging copies
        host_bufs = [h_coords, h_out] + ([] if h_lod is None else [h_lod])
        if all(stf.stf_device_accessible(b) for b in host_bufs):
            def e2e_zero_copy():
                stf.stf_lookup_batch(tex.handle, pe, h_coords, h_lod, n, h_out, None, stream)

            pz, tz = time_steps(torch, e2e_zero_copy, max(3, args.steps // 2), 2, stream)
            extras["e2e_zero_copy"] = {"lookups_per_s": n * len(pz) / (tz / 1000.0),
                                       "how": "pinned host coordinates in and results out, read and "
                                              "written by the lookup kernel over the host link"}
    pe2, te2 = time_steps(torch, e2e_step, max(3, args.steps // 2), 2, stream, dist)
    t_e2e = torch.tensor([te2], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t_e2e, op=dist.ReduceOp.MAX)
    e2e_value = n * world * len(pe2) / (float(t_e2e.item()) / 1000.0)

    if dist is not None:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return 0

    hbm, peak_kind = peaks()
    algo = ALGO_BYTES[(w["name"], "stochastic")]
    avg_launch_ms = statistics.mean(per)
    achieved = algo * n / (avg_launch_ms / 1000.0) / 1e9
    traffic = ncu_traffic(w["name"], filt)
    line = {
        "metric": "filtered lookups/s (stochastic, %s)" % filt,
        "value": value, "unit": "lookups/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        # the filter's arithmetic is float32; the neural decode's MMAs take binary16
        # operands (float32 accumulation)
        "dtype": "f16" if w["name"] == "neural" else "f32",
        "data": "synthetic",
        "config": {"workload": w["desc"], "filter": filt, "queries_per_step": n,
                   "texel_format": TEXEL_FORMAT.get(w["name"], "fp32"),
                   "l2": "inputs larger than L2 (query+output arrays %d MB per step)"
                         % ((w["coords"].nbytes + n * C * 4) // 10**6),
                   "parallelism": "replica per GPU" if world > 1 else "single GPU"},
        "ms_best": min(per), "ms_p50": pct(per, 50), "ms_p99": pct(per, 99),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "algorithmic_bytes_per_lookup": algo, "peak_source": peak_kind},
        "e2e": {"value": e2e_value, "unit": "lookups/s",
                "h2d_bytes_per_step": int(w["coords"].nbytes + (w["lod"].nbytes if lod is not None else 0)),
                "d2h_bytes_per_step": int(n * C * 4)},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "extras": extras,
    }
    if w["name"] == "neural":
        flops = 2 * (8 * 64 + 64 * 64 + 64 * 7)
        tflops = flops * n / (avg_launch_ms / 1000.0) / 1e12
        line["roofline_tensor"] = {"bound": "tensor", "achieved": tflops, "peak": bf16_peak(),
                                   "unit": "TFLOP/s", "frac": tflops / bf16_peak(),
                                   "flops_per_lookup": flops,
                                   "path": "tcgen05.mma kind::f16 (M = 128, binary16 operands, float32 "
                                           "accumulators in tensor memory)"}
        line["config"]["train"] = {"steps": args.train_steps, "batch": 1 << 16,
                                   "loss_first_last": w.get("train_loss")}
        line["config"]["level_mode"] = "nearest (one decode vs four)"
    if not args.no_cpu_baseline and world == 1:     # the CPU baseline is an N = 1 figure
        if w["name"] == "neural":
            p_, z_ = tex.read()
            w["trained_params"], w["trained_latents"] = p_.cpu().numpy(), z_.cpu().numpy()
        ns = min(n, (1 << 22) if w["name"].startswith("sparse") or w["name"] == "neural" else (1 << 24))
        rate, dt, cores = cpu_oracle_rate(w, filt, ns)
        line["cpu_baseline"] = {"value": rate, "unit": "lookups/s", "cores": cores, "kind": "oracle",
                                "sample": "first %d queries of the workload, stochastic %s, "
                                          "%.1f s on %d processes" % (ns, filt, dt, cores)}
        # the same oracle, untimed: the error of the stored texture format
        line["storage_error_vs_fp64_oracle"] = {w["name"]: storage_error(
            stf, torch, w, tex, filt, stream, level_mode=level_mode)}
        for sw, stex in sparse_extra:
            line["storage_error_vs_fp64_oracle"][sw["name"]] = storage_error(stf, torch, sw, stex, filt, stream)
        if w["name"] == "tex2d":
            # the same 2D texture stored in FP16
            t16 = stf.Texture(stf.KIND_TEX2D, w["values"], dims=w["dims"], channels=4, fmt=stf.FMT_F16)
            line["storage_error_vs_fp64_oracle"]["tex2d_fp16"] = storage_error(stf, torch, w, t16, filt, stream)
            t16.close()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    tex.close()
    for _, stex in sparse_extra:
        stex.close()
    return 0


def sparse_extras(stf, torch, args, extras, stream):
    """The largest configuration beside the default one: the sparse 2048^3 cloud
    (FP32 leaves and E4M3 leaves with FP32 leaf scales), 2048x2048 rays x 16 steps
    (67,108,864 queries), stochastic and deterministic tricubic B-spline, each with
    its lookups/s, p50/p99 per launch and HBM fraction.  Returns [(workload, texture)]
    for the storage-error leg."""
    hbm_peak, _ = peaks()
    out_list = []
    base = make_workload("sparse")
    coords = torch.from_numpy(base["coords"]).cuda()
    n = coords.shape[0]
    out = torch.empty((n, 1), dtype=torch.float32, device=coords.device)
    # the queries whose B-spline window touches the active leaves' bounding box
    blo = torch.tensor(base["origins"].min(axis=0), device=coords.device, dtype=coords.dtype)
    bhi = torch.tensor(base["origins"].max(axis=0) + 8, device=coords.device, dtype=coords.dtype)
    fl = torch.floor(coords)
    hits = coords[((fl + 2 >= blo) & (fl - 1 < bhi)).all(dim=1)].contiguous()
    nh = hits.shape[0]
    del fl
    for name in ("sparse", "sparse_e4m3"):
        w = dict(base, name=name)
        T = make_texture(stf, w)
        ps = stf.make_params("bspline3", seed=2024)
        pd = stf.make_params("bspline3")
        sto = lambda: stf.stf_lookup_batch(T.handle, ps, coords, None, n, out, None, stream)
        det = lambda: stf.stf_lookup_batch_deterministic(T.handle, pd, coords, None, n, out, stream)
        p1, t1 = time_steps(torch, sto, max(3, args.steps // 2), 2, stream)
        p2, t2 = time_steps(torch, det, max(3, args.steps // 5), 1, stream)
        hit = lambda: stf.stf_lookup_batch(T.handle, ps, hits, None, nh, out, None, stream)
        p3, t3 = time_steps(torch, hit, max(3, args.steps // 2), 2, stream)
        stf.stf_synchronize(T.handle, stream)
        b = ALGO_BYTES[(name, "stochastic")]
        v1 = n * len(p1) / (t1 / 1000.0)
        v2 = n * len(p2) / (t2 / 1000.0)
        key = "sparse_%s_bspline3" % ("e4m3" if name == "sparse_e4m3" else "fp32")
        extras[key] = {"workload": "sparse 2048^3 cloud, %d leaves, %s leaves, 2048x2048 rays x 16 steps "
                                   "(%d queries)" % (len(w["origins"]), TEXEL_FORMAT[name], n),
                       "lookups_per_s": v1, "ms_p50": pct(p1, 50), "ms_p99": pct(p1, 99),
                       "hbm_frac": v1 * b / 1e9 / hbm_peak, "algorithmic_bytes_per_lookup": b,
                       "deterministic_lookups_per_s": v2, "deterministic_ms_p50": pct(p2, 50),
                       "speedup_vs_deterministic": v1 / v2,
                       "hits_only": {"queries": nh, "fraction_of_workload": nh / n,
                                     "lookups_per_s": nh * len(p3) / (t3 / 1000.0),
                                     "hbm_frac": nh * len(p3) / (t3 / 1000.0) * b / 1e9 / hbm_peak}}
        out_list.append((w, T))
    del coords, out, hits
    return out_list


def main():
    args = parse()
    if args.filter is None:
        args.filter = "linear" if args.workload == "neural" else "bspline3"
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "aniso":
        return run_aniso(args)
    if args.workload == "dct":
        return run_dct(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
