"""Python binding of libstf.so, the GB300 stochastic texture filtering library.

The functions carry the C ABI's names (``include/stf.h``) and only marshal
arguments: torch tensors become device pointers, the current torch stream becomes
the CUDA stream.  Every lookup runs in the library's CUDA kernels; if the library
is missing or cannot be loaded the binding raises -- there is no fallback.
"""
import ctypes
import os

from . import build as _build

__all__ = [
    "StfError", "TextureDesc", "LookupParams", "stf_create_texture", "stf_destroy",
    "stf_lookup_batch", "stf_lookup_batch_deterministic", "stf_lookup_accumulate",
    "stf_lookup_batch_binned_noalloc",
    "stf_texture_bytes", "stf_synchronize", "stf_device_accessible", "stf_last_error", "stf_version", "Texture",
    "KIND_TEX2D", "KIND_DENSE3D", "KIND_SPARSE3D", "FMT_F32", "FMT_F16", "FMT_E4M3_SCALED",
    "FILTER_LINEAR", "FILTER_BSPLINE3", "FILTER_CATMULL_ROM", "LEVEL_NEAREST",
    "LEVEL_STOCHASTIC", "library_path", "load", "NeuralDesc", "TrainConfig",
    "stf_create_neural_texture", "stf_neural_gradients", "stf_neural_train", "stf_neural_read",
    "NeuralTexture", "KIND_NEURAL2D", "stf_anisotropic_lod", "stf_lookup_batch_ewa",
    "stf_lookup_batch_ewa_deterministic", "stf_ewa_weight_table", "STF_EWA_MAX_ANISOTROPY",
    "stf_lookup_batch_triplanar", "stf_lookup_batch_triplanar_deterministic", "FMT_DCT6",
]

KIND_TEX2D, KIND_DENSE3D, KIND_SPARSE3D, KIND_NEURAL2D = 0, 1, 2, 3
NEURAL_LATENT, NEURAL_HIDDEN, NEURAL_OUT, NEURAL_PARAMS = 8, 64, 7, 5191
FMT_F32, FMT_F16, FMT_E4M3_SCALED, FMT_DCT6 = 0, 1, 2, 3
FILTER_LINEAR, FILTER_BSPLINE3, FILTER_CATMULL_ROM, FILTER_CATMULL_ROM_POSITIVIZED = 0, 1, 2, 3
FILTER_FIS_LINEAR, FILTER_FIS_BSPLINE3, FILTER_FIS_GAUSSIAN = 4, 5, 6
FIS_MAX_WIDTH = 8.0                  # include/stf.h STF_FIS_MAX_WIDTH
FILTERS = {"linear": FILTER_LINEAR, "bspline3": FILTER_BSPLINE3, "catmull_rom": FILTER_CATMULL_ROM,
           "catmull_rom_positivized": FILTER_CATMULL_ROM_POSITIVIZED,
           "fis_linear": FILTER_FIS_LINEAR, "fis_bspline3": FILTER_FIS_BSPLINE3,
           "fis_gaussian": FILTER_FIS_GAUSSIAN}
LEVEL_NEAREST, LEVEL_STOCHASTIC = 0, 1
STF_NOALLOC_MAX_QUERIES = 1 << 20   # include/stf.h
STF_EWA_MAX_ANISOTROPY = 64.0       # include/stf.h

STATUS = {0: "STF_OK", 1: "STF_ERR_INVALID_ARGUMENT", 2: "STF_ERR_INVALID_HANDLE",
          3: "STF_ERR_OUT_OF_MEMORY", 4: "STF_ERR_UNSUPPORTED", 5: "STF_ERR_CUDA",
          6: "STF_ERR_DEVICE_ASSERT", 7: "STF_ERR_BUDGET"}


class StfError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class TextureDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("format", ctypes.c_int32),
                ("dims", ctypes.c_int32 * 3), ("channels", ctypes.c_int32),
                ("mip_levels", ctypes.c_int32), ("generate_mips", ctypes.c_int32),
                ("data_on_device", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("data", ctypes.c_void_p), ("leaf_origins", ctypes.c_void_p),
                ("num_leaves", ctypes.c_int64), ("background", ctypes.c_float),
                ("reserved1", ctypes.c_int32)]


class LookupParams(ctypes.Structure):
    _fields_ = [("filter", ctypes.c_int32), ("level_mode", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("query_offset", ctypes.c_uint64),
                ("sample_index", ctypes.c_uint32), ("bin_queries", ctypes.c_int32),
                ("reuse_xi", ctypes.c_int32), ("filter_width", ctypes.c_float)]


class NeuralDesc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("latent_levels", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("data_on_device", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("latents", ctypes.c_void_p), ("params", ctypes.c_void_p),
                ("fallback", ctypes.c_void_p)]


class TrainConfig(ctypes.Structure):
    _fields_ = [("lr_latent", ctypes.c_float), ("lr_params", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("batch", ctypes.c_int32), ("seed", ctypes.c_uint64)]


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libstf.so (building it first if asked and needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise OSError("libstf.so is missing: run paper_2305_05810_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB)
    P, I32, I64, VP = ctypes.POINTER, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    lib.stf_create_texture.argtypes = [P(TextureDesc), VP, P(VP)]
    lib.stf_destroy.argtypes = [VP]
    lib.stf_lookup_batch.argtypes = [VP, P(LookupParams), VP, VP, I64, VP, VP, VP]
    lib.stf_lookup_batch_deterministic.argtypes = [VP, P(LookupParams), VP, VP, I64, VP, VP]
    lib.stf_lookup_batch_binned_noalloc.argtypes = [VP, P(LookupParams), VP, VP, I64, VP, VP, VP]
    lib.stf_lookup_accumulate.argtypes = [VP, P(LookupParams), VP, VP, I64, I32, VP, VP, VP]
    lib.stf_texture_bytes.argtypes = [VP, P(I64)]
    lib.stf_synchronize.argtypes = [VP, VP]
    lib.stf_device_accessible.argtypes = [VP, P(I32)]
    lib.stf_last_error.restype = ctypes.c_char_p
    lib.stf_last_error.argtypes = []
    lib.stf_version.restype = I32
    lib.stf_create_neural_texture.argtypes = [P(NeuralDesc), VP, P(VP)]
    lib.stf_neural_gradients.argtypes = [VP, VP, I64, VP, VP, VP, VP, VP]
    lib.stf_neural_train.argtypes = [VP, VP, P(TrainConfig), I32, VP, VP]
    lib.stf_neural_read.argtypes = [VP, VP, VP, VP]
    F32 = ctypes.c_float
    lib.stf_anisotropic_lod.argtypes = [VP, VP, I64, F32, VP, VP]
    lib.stf_lookup_batch_ewa.argtypes = [VP, P(LookupParams), VP, VP, I64, F32, VP, VP, VP]
    lib.stf_lookup_batch_ewa_deterministic.argtypes = [VP, P(LookupParams), VP, VP, I64, F32, VP, VP]
    lib.stf_ewa_weight_table.argtypes = [VP]
    lib.stf_lookup_batch_triplanar.argtypes = [VP, P(LookupParams), VP, VP, VP, I64, F32, VP, VP, VP]
    lib.stf_lookup_batch_triplanar_deterministic.argtypes = [VP, P(LookupParams), VP, VP, VP, I64, F32,
                                                             VP, VP]
    lib.stf_debug_fail_allocation.argtypes = [I64]
    lib.stf_debug_fail_allocation.restype = None
    for f in ("stf_create_texture", "stf_destroy", "stf_lookup_batch",
              "stf_lookup_batch_deterministic", "stf_lookup_accumulate", "stf_texture_bytes",
              "stf_synchronize", "stf_device_accessible", "stf_lookup_batch_binned_noalloc",
              "stf_create_neural_texture",
              "stf_neural_gradients", "stf_neural_train", "stf_neural_read", "stf_anisotropic_lod",
              "stf_lookup_batch_ewa", "stf_lookup_batch_ewa_deterministic", "stf_ewa_weight_table",
              "stf_lookup_batch_triplanar", "stf_lookup_batch_triplanar_deterministic"):
        getattr(lib, f).restype = I32
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise StfError(status, load().stf_last_error().decode())


def _ptr(x):
    """Device/host address of a tensor, an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def stf_last_error():
    return load().stf_last_error().decode()


def stf_version():
    return load().stf_version()


def stf_create_texture(desc, stream=None):
    h = ctypes.c_void_p()
    _check(load().stf_create_texture(ctypes.byref(desc), _stream(stream), ctypes.byref(h)))
    return h.value


def stf_create_neural_texture(desc, stream=None):
    h = ctypes.c_void_p()
    _check(load().stf_create_neural_texture(ctypes.byref(desc), _stream(stream), ctypes.byref(h)))
    return h.value


def stf_neural_gradients(tex, texels, batch, target_rows, param_grads=None, latent_grads=None,
                         loss=None, stream=None):
    _check(load().stf_neural_gradients(tex, _ptr(texels), int(batch), _ptr(target_rows),
                                       _ptr(param_grads), _ptr(latent_grads), _ptr(loss),
                                       _stream(stream)))


def stf_neural_train(tex, target, config, steps, loss_per_step=None, stream=None):
    _check(load().stf_neural_train(tex, _ptr(target), ctypes.byref(config), int(steps),
                                   _ptr(loss_per_step), _stream(stream)))


def stf_neural_read(tex, params=None, latents=None, stream=None):
    _check(load().stf_neural_read(tex, _ptr(params), _ptr(latents), _stream(stream)))


def stf_destroy(tex):
    _check(load().stf_destroy(tex))


def stf_lookup_batch(tex, params, coords, lod, n, out, taps=None, stream=None):
    _check(load().stf_lookup_batch(tex, ctypes.byref(params), _ptr(coords), _ptr(lod), int(n),
                                   _ptr(out), _ptr(taps), _stream(stream)))


def stf_lookup_batch_binned_noalloc(tex, params, coords, lod, n, out, taps=None, stream=None):
    _check(load().stf_lookup_batch_binned_noalloc(tex, ctypes.byref(params), _ptr(coords), _ptr(lod),
                                                  int(n), _ptr(out), _ptr(taps), _stream(stream)))


def stf_lookup_batch_deterministic(tex, params, coords, lod, n, out, stream=None):
    _check(load().stf_lookup_batch_deterministic(tex, ctypes.byref(params), _ptr(coords),
                                                 _ptr(lod), int(n), _ptr(out), _stream(stream)))


def stf_lookup_accumulate(tex, params, coords, lod, n, n_samples, d_sum, d_sumsq, stream=None):
    _check(load().stf_lookup_accumulate(tex, ctypes.byref(params), _ptr(coords), _ptr(lod),
                                        int(n), int(n_samples), _ptr(d_sum), _ptr(d_sumsq),
                                        _stream(stream)))


def stf_anisotropic_lod(tex, grad, n, max_anisotropy, lod, stream=None):
    _check(load().stf_anisotropic_lod(tex, _ptr(grad), int(n), float(max_anisotropy), _ptr(lod),
                                      _stream(stream)))


def stf_lookup_batch_ewa(tex, params, uv, grad, n, max_anisotropy, out, taps=None, stream=None):
    _check(load().stf_lookup_batch_ewa(tex, ctypes.byref(params), _ptr(uv), _ptr(grad), int(n),
                                       float(max_anisotropy), _ptr(out), _ptr(taps), _stream(stream)))


def stf_lookup_batch_ewa_deterministic(tex, params, uv, grad, n, max_anisotropy, out, stream=None):
    _check(load().stf_lookup_batch_ewa_deterministic(tex, ctypes.byref(params), _ptr(uv), _ptr(grad),
                                                     int(n), float(max_anisotropy), _ptr(out),
                                                     _stream(stream)))


def stf_lookup_batch_triplanar(tex, params, pos, normal, lod, n, scale, out, taps=None, stream=None):
    _check(load().stf_lookup_batch_triplanar(tex, ctypes.byref(params), _ptr(pos), _ptr(normal), _ptr(lod),
                                             int(n), float(scale), _ptr(out), _ptr(taps), _stream(stream)))


def stf_lookup_batch_triplanar_deterministic(tex, params, pos, normal, lod, n, scale, out, stream=None):
    _check(load().stf_lookup_batch_triplanar_deterministic(tex, ctypes.byref(params), _ptr(pos),
                                                           _ptr(normal), _ptr(lod), int(n), float(scale),
                                                           _ptr(out), _stream(stream)))


def stf_ewa_weight_table():
    buf = (ctypes.c_float * 128)()
    _check(load().stf_ewa_weight_table(ctypes.addressof(buf)))
    return list(buf)


def stf_texture_bytes(tex):
    b = ctypes.c_int64()
    _check(load().stf_texture_bytes(tex, ctypes.byref(b)))
    return b.value


def stf_device_accessible(x):
    """True if the current device can address the tensor (or address) x at that same
    address: device memory, or pinned host memory mapped into the device's space."""
    v = ctypes.c_int32()
    _check(load().stf_device_accessible(_ptr(x), ctypes.byref(v)))
    return bool(v.value)


def stf_synchronize(tex, stream=None):
    _check(load().stf_synchronize(tex, _stream(stream)))


def make_params(filter="bspline3", seed=0, sample_index=0, query_offset=0, level_mode=LEVEL_STOCHASTIC,
                bin_queries=False, reuse_xi=False, width=0.0):
    f = FILTERS[filter] if isinstance(filter, str) else int(filter)
    return LookupParams(filter=f, level_mode=level_mode, seed=seed, query_offset=query_offset,
                        sample_index=sample_index, bin_queries=int(bin_queries),
                        reuse_xi=int(reuse_xi), filter_width=float(width))


class Texture:
    """Owning wrapper around a texture handle, for tensors on the current device."""

    def __init__(self, kind, data, *, fmt=FMT_F32, dims=(1, 1, 1), channels=1, mip_levels=1,
                 generate_mips=False, leaf_origins=None, background=0.0, stream=None):
        import torch
        data = data if isinstance(data, torch.Tensor) else torch.as_tensor(data)
        data = data.to(torch.float32).contiguous()
        self._keep = [data]
        desc = TextureDesc(kind=kind, format=fmt, channels=channels, mip_levels=mip_levels,
                           generate_mips=int(generate_mips), data_on_device=int(data.is_cuda),
                           data=data.data_ptr(), background=background)
        desc.dims[:] = list(dims)
        if leaf_origins is not None:
            lo = leaf_origins if isinstance(leaf_origins, torch.Tensor) else torch.as_tensor(leaf_origins)
            lo = lo.to(device=data.device, dtype=torch.int32).contiguous()
            self._keep.append(lo)
            desc.leaf_origins = lo.data_ptr()
            desc.num_leaves = lo.shape[0]
        self.kind, self.channels = kind, channels
        self.handle = stf_create_texture(desc, stream)
        self._keep = None

    def close(self):
        if self.handle is not None:
            stf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nbytes(self):
        return stf_texture_bytes(self.handle)

    def lookup(self, coords, lod=None, *, out=None, taps=None, stream=None, **params):
        import torch
        n = coords.shape[0]
        if out is None:
            out = torch.empty((n, self.channels), dtype=torch.float32, device=coords.device)
        stf_lookup_batch(self.handle, make_params(**params), coords, lod, n, out, taps, stream)
        return out

    def lookup_deterministic(self, coords, lod=None, *, out=None, stream=None, **params):
        import torch
        n = coords.shape[0]
        if out is None:
            out = torch.empty((n, self.channels), dtype=torch.float32, device=coords.device)
        stf_lookup_batch_deterministic(self.handle, make_params(**params), coords, lod, n, out, stream)
        return out

    def accumulate(self, coords, n_samples, lod=None, *, stream=None, **params):
        import torch
        n = coords.shape[0]
        s = torch.empty((n, self.channels), dtype=torch.float64, device=coords.device)
        s2 = torch.empty_like(s)
        stf_lookup_accumulate(self.handle, make_params(**params), coords, lod, n, n_samples, s, s2,
                              stream)
        return s, s2


    def lookup_ewa(self, uv, grad, max_anisotropy=STF_EWA_MAX_ANISOTROPY, *, out=None, taps=None,
                   stream=None, **params):
        import torch
        n = uv.shape[0]
        if out is None:
            out = torch.empty((n, self.channels), dtype=torch.float32, device=uv.device)
        stf_lookup_batch_ewa(self.handle, make_params(**params), uv, grad, n, max_anisotropy, out,
                             taps, stream)
        return out

    def lookup_ewa_deterministic(self, uv, grad, max_anisotropy=STF_EWA_MAX_ANISOTROPY, *, out=None,
                                 stream=None, **params):
        import torch
        n = uv.shape[0]
        if out is None:
            out = torch.empty((n, self.channels), dtype=torch.float32, device=uv.device)
        stf_lookup_batch_ewa_deterministic(self.handle, make_params(**params), uv, grad, n,
                                           max_anisotropy, out, stream)
        return out

    def lookup_triplanar(self, pos, normal, scale=1.0, lod=None, *, out=None, taps=None, stream=None,
                         **params):
        import torch
        n = pos.shape[0]
        if out is None:
            out = torch.empty((n, self.channels), dtype=torch.float32, device=pos.device)
        stf_lookup_batch_triplanar(self.handle, make_params(**params), pos, normal, lod, n, scale, out,
                                   taps, stream)
        return out

    def lookup_triplanar_deterministic(self, pos, normal, scale=1.0, lod=None, *, out=None, stream=None,
                                       **params):
        import torch
        n = pos.shape[0]
        if out is None:
            out = torch.empty((n, self.channels), dtype=torch.float32, device=pos.device)
        stf_lookup_batch_triplanar_deterministic(self.handle, make_params(**params), pos, normal, lod, n,
                                                 scale, out, stream)
        return out

    def anisotropic_lod(self, grad, max_anisotropy=STF_EWA_MAX_ANISOTROPY, *, out=None, stream=None):
        import torch
        n = grad.shape[0]
        if out is None:
            out = torch.empty((n,), dtype=torch.float32, device=grad.device)
        stf_anisotropic_lod(self.handle, grad, n, max_anisotropy, out, stream)
        return out


class NeuralTexture(Texture):
    """Owning wrapper around a neural texture (latent levels + decoder MLP)."""

    def __init__(self, width, height, latent_levels, levels, latents, params, fallback=None,
                 stream=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        f32 = lambda a: (a if isinstance(a, torch.Tensor) else torch.as_tensor(a)).to(dev, torch.float32).contiguous()
        lat, par = f32(latents), f32(params)
        fb = None if fallback is None else f32(fallback)
        desc = NeuralDesc(width=width, height=height, latent_levels=latent_levels, levels=levels,
                          data_on_device=1, latents=lat.data_ptr(), params=par.data_ptr(),
                          fallback=None if fb is None else fb.data_ptr())
        self.kind, self.channels = KIND_NEURAL2D, NEURAL_OUT
        self.n_latent_texels = lat.numel() // NEURAL_LATENT
        self.handle = stf_create_neural_texture(desc, stream)

    def gradients(self, texels, targets, stream=None):
        import torch
        n = texels.shape[0]
        pg = torch.empty(NEURAL_PARAMS, dtype=torch.float32, device=texels.device)
        lg = torch.empty((n, NEURAL_LATENT), dtype=torch.float32, device=texels.device)
        loss = torch.empty(1, dtype=torch.float32, device=texels.device)
        stf_neural_gradients(self.handle, texels, n, targets, pg, lg, loss, stream)
        return pg, lg, loss

    def train(self, target, steps, batch=65536, lr_latent=1e-2, lr_params=1e-3, seed=0, stream=None):
        import torch
        cfg = TrainConfig(lr_latent=lr_latent, lr_params=lr_params, beta1=0.9, beta2=0.999,
                          eps=1e-8, batch=batch, seed=seed)
        losses = torch.empty(max(1, steps), dtype=torch.float32, device=target.device)
        stf_neural_train(self.handle, target, cfg, steps, losses, stream)
        return losses[:steps]

    def read(self, stream=None):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        p = torch.empty(NEURAL_PARAMS, dtype=torch.float32, device=dev)
        z = torch.empty((self.n_latent_texels, NEURAL_LATENT), dtype=torch.float32, device=dev)
        stf_neural_read(self.handle, p, z, stream)
        return p, z
