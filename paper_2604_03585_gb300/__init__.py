"""Python binding of libsar, the GB300 (sm_103a) kernel-fused SAR Range-Doppler
compression library.

This module only marshals arguments: every step of the compression runs in
the CUDA kernels of ``libsar.so`` (built in-tree from ``csrc/`` by
``build.py``).  The function names are those of the C-ABI in
``include/sar.h``.  If the library is missing, importing this package raises
ImportError; there is no fallback of any kind.

Tensors are torch tensors of dtype complex64 on the current CUDA device
(contiguous); streams default to torch's current stream.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsar.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsar.so is not built ({LIB_PATH}); run paper_2604_03585_gb300/build.py "
                      "or __graft_entry__.build() first")

_lib = ctypes.CDLL(LIB_PATH)

SAR_OK, SAR_ERR_INVALID_ARG, SAR_ERR_UNSUPPORTED, SAR_ERR_OUT_OF_MEMORY, SAR_ERR_CUDA, SAR_ERR_TIMEOUT = range(6)
SAR_PREC_FP32, SAR_PREC_FP16X2, SAR_PREC_BF16X2, SAR_PREC_BF16X3 = 0, 1, 2, 3
SAR_PLAN_UNFOLDED_CORNER_TURN = 1
SAR_PLAN_OUT_AZ_MAJOR = 2
SAR_BATCH_EXACT_AZIMUTH = 1
SAR_BATCH_MULTI_KERNEL = 2
SAR_BATCH_AUTOTUNE = 4
SAR_TUNE_FUSED, SAR_TUNE_RANGE_CT = 0, 1
SAR_SERVE_OPEN_LOOP, SAR_SERVE_CLOSED_LOOP = 0, 1

STATUS_NAMES = {0: "SAR_OK", 1: "SAR_ERR_INVALID_ARG", 2: "SAR_ERR_UNSUPPORTED",
                3: "SAR_ERR_OUT_OF_MEMORY", 4: "SAR_ERR_CUDA", 5: "SAR_ERR_TIMEOUT"}

# every entry point declared in include/sar.h
EXPORTS = ("sar_plan_create", "sar_plan_destroy", "sar_range_compress", "sar_corner_turn",
           "sar_azimuth_compress", "sar_rda_process", "sar_range_compress_oop", "sar_range_compress_ct", "sar_rda_process_oop",
           "sar_range_compress_unfused", "sar_azimuth_compress_unfused", "sar_rda_process_unfused",
           "sar_plan_set_geometry", "sar_rcmc", "sar_rda_full",
           "sar_rda_process_host", "sar_rda_process_host_n", "sar_make_lfm_spectrum", "sar_simulate_echo",
           "sar_fft_lines", "sar_fft_lines_static", "sar_transpose", "sar_schedule_count", "sar_schedule_get",
           "sar_set_preferred_schedule", "sar_set_corner_turn_variant", "sar_set_split_engine", "sar_plan_create_ex", "sar_plan_get_schedules", "sar_plan_folds_corner_turn", "sar_autotune",
           "sar_plan_status", "sar_batch_create", "sar_batch_run", "sar_batch_info", "sar_batch_status",
           "sar_batch_destroy", "sar_server_create", "sar_server_run", "sar_server_destroy",
           "sar_sync", "sar_last_error", "sar_version")


class sar_schedule_desc(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("n", ctypes.c_int32), ("e", ctypes.c_int32),
                ("r1", ctypes.c_int32), ("r2", ctypes.c_int32), ("r3", ctypes.c_int32),
                ("lines_per_block", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32), ("cluster_blocks", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: (getattr(self, f).decode() if f == "name" else getattr(self, f)) for f, _ in self._fields_}


class sar_strip(ctypes.Structure):
    _fields_ = [("n_range", ctypes.c_int64), ("n_az", ctypes.c_int64), ("raw", ctypes.c_void_p),
                ("image", ctypes.c_void_p), ("range_spectrum", ctypes.c_void_p), ("az_spectrum", ctypes.c_void_p)]


class sar_batch_info_t(ctypes.Structure):
    _fields_ = [("strips", ctypes.c_int64), ("samples", ctypes.c_int64), ("work_bytes", ctypes.c_int64),
                ("kernels_per_run", ctypes.c_int32), ("range_classes", ctypes.c_int32),
                ("azimuth_classes", ctypes.c_int32)]


class sar_server_config(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("n_range", ctypes.POINTER(ctypes.c_int64)), ("n_az", ctypes.POINTER(ctypes.c_int64)),
                ("pool", ctypes.POINTER(ctypes.c_void_p)), ("range_spectrum", ctypes.POINTER(ctypes.c_void_p)),
                ("az_spectrum", ctypes.POINTER(ctypes.c_void_p)), ("hbm_budget_bytes", ctypes.c_int64),
                ("backfill_s", ctypes.c_double), ("size_priority", ctypes.c_int32), ("aging_s", ctypes.c_double)]


class sar_request(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("size_class", ctypes.c_int32), ("output", ctypes.c_void_p)]


class sar_request_result(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("status", ctypes.c_int32)]


class sar_filters(ctypes.Structure):
    _fields_ = [("range_spectrum", ctypes.c_void_p), ("az_spectrum", ctypes.c_void_p),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32)]


_i64, _vp, _int, _dbl = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_SIGS = {
    "sar_plan_create": [_i64, _i64, ctypes.POINTER(sar_filters), ctypes.POINTER(_vp)],
    "sar_plan_destroy": [_vp],
    "sar_range_compress": [_vp, _vp, _vp],
    "sar_corner_turn": [_vp, _vp, _vp, _vp],
    "sar_azimuth_compress": [_vp, _vp, _vp],
    "sar_rda_process": [_vp, _vp, _vp, _vp],
    "sar_range_compress_oop": [_vp, _vp, _vp, _vp],
    "sar_range_compress_ct": [_vp, _vp, _vp, _vp],
    "sar_range_compress_unfused": [_vp, _vp, _vp],
    "sar_azimuth_compress_unfused": [_vp, _vp, _vp],
    "sar_rda_process_unfused": [_vp, _vp, _vp, _vp],
    "sar_plan_set_geometry": [_vp, _dbl, _dbl, _dbl, ctypes.c_int32],
    "sar_rcmc": [_vp, _vp, _vp, _vp],
    "sar_rda_full": [_vp, _vp, _vp, _vp, _vp],
    "sar_rda_process_oop": [_vp, _vp, _vp, _vp, _vp],
    "sar_rda_process_host": [_vp, _vp, _vp, _vp],
    "sar_rda_process_host_n": [_vp, ctypes.c_int32, _vp, _vp, _vp],
    "sar_make_lfm_spectrum": [_i64, _i64, _dbl, _vp, _vp],
    "sar_simulate_echo": [_i64, _i64, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, _i64, _dbl, _i64, _dbl, _dbl,
                          ctypes.c_uint64, _vp, _vp],
    "sar_fft_lines": [_i64, _i64, _vp, _vp, _int, _vp],
    "sar_fft_lines_static": [_i64, _i64, _vp, _vp, _int, _vp],
    "sar_transpose": [_i64, _i64, _vp, _vp, _vp],
    "sar_sync": [_vp],
    "sar_plan_status": [_vp, _vp],
    "sar_batch_create": [ctypes.POINTER(sar_strip), ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(_vp)],
    "sar_batch_run": [_vp, _vp],
    "sar_batch_status": [_vp, _vp],
    "sar_batch_info": [_vp, ctypes.POINTER(sar_batch_info_t)],
    "sar_batch_destroy": [_vp],
    "sar_server_create": [ctypes.POINTER(sar_server_config), ctypes.POINTER(_vp)],
    "sar_server_run": [_vp, ctypes.POINTER(sar_request), ctypes.c_int32, ctypes.c_int32,
                       ctypes.POINTER(sar_request_result)],
    "sar_server_destroy": [_vp],
    "sar_schedule_get": [ctypes.c_int32, ctypes.POINTER(sar_schedule_desc)],
    "sar_set_preferred_schedule": [ctypes.c_char_p],
    "sar_set_corner_turn_variant": [ctypes.c_int32],
    "sar_set_split_engine": [ctypes.c_int32],
    "sar_plan_create_ex": [_i64, _i64, ctypes.POINTER(sar_filters), ctypes.c_char_p, ctypes.c_char_p,
                           ctypes.POINTER(_vp)],
    "sar_plan_get_schedules": [_vp, ctypes.POINTER(sar_schedule_desc), ctypes.POINTER(sar_schedule_desc)],
    "sar_autotune": [_i64, _i64, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.POINTER(sar_schedule_desc),
                     ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), ctypes.c_int32],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.sar_plan_folds_corner_turn.restype = ctypes.c_int32
_lib.sar_plan_folds_corner_turn.argtypes = [_vp]
_lib.sar_schedule_count.restype = ctypes.c_int32
_lib.sar_schedule_count.argtypes = []
_lib.sar_last_error.restype = ctypes.c_char_p
_lib.sar_version.restype = ctypes.c_char_p


class SarError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


def _check(st: int) -> None:
    if st != SAR_OK:
        raise SarError(st, _lib.sar_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x):
    """Device (or host) address of a tensor / numpy array / raw int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def library() -> ctypes.CDLL:
    return _lib


def sar_version() -> str:
    return _lib.sar_version().decode()


def sar_last_error() -> str:
    return _lib.sar_last_error().decode()


class Plan:
    """An opaque sar_plan handle (destroyed with the object or explicitly)."""

    def __init__(self, handle: int, n_range: int, n_az: int):
        self.handle = handle
        self.n_range = n_range
        self.n_az = n_az

    def destroy(self) -> None:
        if self.handle:
            _check(_lib.sar_plan_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sar_plan_create(n_range: int, n_az: int, range_spectrum, az_spectrum, precision: int = SAR_PREC_FP32,
                    flags: int = 0) -> Plan:
    f = sar_filters(_ptr(range_spectrum), _ptr(az_spectrum), precision, flags)
    h = _vp()
    _check(_lib.sar_plan_create(n_range, n_az, ctypes.byref(f), ctypes.byref(h)))
    return Plan(h.value, n_range, n_az)


def sar_plan_create_ex(n_range: int, n_az: int, range_spectrum, az_spectrum, range_schedule=None,
                       az_schedule=None, precision: int = SAR_PREC_FP32, flags: int = 0) -> Plan:
    f = sar_filters(_ptr(range_spectrum), _ptr(az_spectrum), precision, flags)
    h = _vp()
    enc = lambda x: None if x is None else x.encode()
    _check(_lib.sar_plan_create_ex(n_range, n_az, ctypes.byref(f), enc(range_schedule), enc(az_schedule),
                                   ctypes.byref(h)))
    return Plan(h.value, n_range, n_az)


def sar_plan_folds_corner_turn(plan) -> bool:
    return bool(_lib.sar_plan_folds_corner_turn(_h(plan)))


def sar_plan_get_schedules(plan) -> tuple:
    r, a = sar_schedule_desc(), sar_schedule_desc()
    _check(_lib.sar_plan_get_schedules(_h(plan), ctypes.byref(r), ctypes.byref(a)))
    return r.as_dict(), a.as_dict()


def sar_schedule_count() -> int:
    return int(_lib.sar_schedule_count())


def sar_schedule_get(index: int) -> dict:
    d = sar_schedule_desc()
    _check(_lib.sar_schedule_get(index, ctypes.byref(d)))
    return d.as_dict()


def schedules(n: int | None = None) -> list:
    out = [sar_schedule_get(i) for i in range(sar_schedule_count())]
    return [d for d in out if n is None or d["n"] == n]


def sar_set_preferred_schedule(name: str) -> None:
    _check(_lib.sar_set_preferred_schedule(name.encode()))


def sar_set_corner_turn_variant(variant: int) -> None:
    _check(_lib.sar_set_corner_turn_variant(variant))


def sar_set_split_engine(engine: int) -> None:
    """Engine of split-precision plans: 0 tcgen05.mma (TMEM accumulators), 1 mma.sync."""
    _check(_lib.sar_set_split_engine(engine))


def sar_autotune(n: int, n_lines: int, reps: int = 20, stream=None, kind: int = SAR_TUNE_FUSED) -> tuple:
    """Time every schedule of length n for one kind of kernel; returns (best
    schedule, best ms, {schedule name: median ms}), leaving out schedules
    without that kind of kernel."""
    d = sar_schedule_desc()
    ms = ctypes.c_float()
    cands = schedules(n)
    arr = (ctypes.c_float * max(1, len(cands)))()
    _check(_lib.sar_autotune(n, n_lines, reps, kind, _stream(stream), ctypes.byref(d), ctypes.byref(ms), arr,
                             len(cands)))
    return d.as_dict(), float(ms.value), {c["name"]: float(arr[i]) for i, c in enumerate(cands) if arr[i] > 0}


def sar_plan_destroy(plan: Plan) -> None:
    plan.destroy()


def _h(obj):
    return obj.handle if hasattr(obj, "handle") else obj


def sar_range_compress(plan, data, stream=None) -> None:
    _check(_lib.sar_range_compress(_h(plan), _ptr(data), _stream(stream)))


def sar_corner_turn(plan, inp, out, stream=None) -> None:
    _check(_lib.sar_corner_turn(_h(plan), _ptr(inp), _ptr(out), _stream(stream)))


def sar_azimuth_compress(plan, data, stream=None) -> None:
    _check(_lib.sar_azimuth_compress(_h(plan), _ptr(data), _stream(stream)))


def sar_rda_process(plan, raw, image, stream=None) -> None:
    _check(_lib.sar_rda_process(_h(plan), _ptr(raw), _ptr(image), _stream(stream)))


def sar_range_compress_oop(plan, inp, out, stream=None) -> None:
    _check(_lib.sar_range_compress_oop(_h(plan), _ptr(inp), _ptr(out), _stream(stream)))


def sar_range_compress_ct(plan, raw, image, stream=None) -> None:
    _check(_lib.sar_range_compress_ct(_h(plan), _ptr(raw), _ptr(image), _stream(stream)))


def sar_range_compress_unfused(plan, data, stream=None) -> None:
    _check(_lib.sar_range_compress_unfused(_h(plan), _ptr(data), _stream(stream)))


def sar_azimuth_compress_unfused(plan, data, stream=None) -> None:
    _check(_lib.sar_azimuth_compress_unfused(_h(plan), _ptr(data), _stream(stream)))


def sar_rda_process_unfused(plan, raw, image, stream=None) -> None:
    _check(_lib.sar_rda_process_unfused(_h(plan), _ptr(raw), _ptr(image), _stream(stream)))


def sar_plan_set_geometry(plan, kappa: float, v_s: float, r_near: float, rcmc_taps: int = 16) -> None:
    _check(_lib.sar_plan_set_geometry(_h(plan), float(kappa), float(v_s), float(r_near), int(rcmc_taps)))


def sar_rcmc(plan, data_in, data_out, stream=None) -> None:
    _check(_lib.sar_rcmc(_h(plan), _ptr(data_in), _ptr(data_out), _stream(stream)))


def sar_rda_full(plan, raw, work, image, stream=None) -> None:
    _check(_lib.sar_rda_full(_h(plan), _ptr(raw), _ptr(work), _ptr(image), _stream(stream)))


def sar_rda_process_oop(plan, raw, work, image, stream=None) -> None:
    _check(_lib.sar_rda_process_oop(_h(plan), _ptr(raw), _ptr(work), _ptr(image), _stream(stream)))


def sar_rda_process_host(plan, raw_host, image_host, stream=None) -> None:
    _check(_lib.sar_rda_process_host(_h(plan), _ptr(raw_host), _ptr(image_host), _stream(stream)))


def sar_rda_process_host_n(plan, raws_host, images_host, stream=None) -> None:
    """Scenes raws_host[q] -> images_host[q] (host buffers) in one call."""
    if len(raws_host) != len(images_host):
        raise ValueError("one image per echo")
    n = len(raws_host)
    raws = (ctypes.c_void_p * max(n, 1))(*[_ptr(r) for r in raws_host])
    imgs = (ctypes.c_void_p * max(n, 1))(*[_ptr(m) for m in images_host])
    _check(_lib.sar_rda_process_host_n(_h(plan), n, raws, imgs, _stream(stream)))


def sar_make_lfm_spectrum(n: int, n_chirp: int, tbp: float, out, stream=None) -> None:
    _check(_lib.sar_make_lfm_spectrum(n, n_chirp, float(tbp), _ptr(out), _stream(stream)))


def sar_simulate_echo(n_az: int, n_range: int, targets, range_chirp, az_chirp, snr_db, seed: int, out,
                      stream=None) -> None:
    """targets: [(a0, r0), ...]; range_chirp / az_chirp: (n_c, tbp); snr_db None: no noise."""
    flat = (ctypes.c_int64 * max(1, 2 * len(targets)))(*[int(v) for t in targets for v in t])
    _check(_lib.sar_simulate_echo(n_az, n_range, flat, len(targets), int(range_chirp[0]), float(range_chirp[1]),
                                  int(az_chirp[0]), float(az_chirp[1]),
                                  float("nan") if snr_db is None else float(snr_db), seed, _ptr(out),
                                  _stream(stream)))


def sar_fft_lines(n: int, n_lines: int, inp, out, inverse: bool = False, stream=None) -> None:
    _check(_lib.sar_fft_lines(n, n_lines, _ptr(inp), _ptr(out), 1 if inverse else 0, _stream(stream)))


def sar_fft_lines_static(n: int, n_lines: int, inp, out, inverse: bool = False, stream=None) -> None:
    """sar_fft_lines for callers that must not have device memory allocated
    for them (stream capture, fixed-footprint real-time code, pool-owned
    memory): its twiddles live in a fixed 256 KiB device array shared by all
    calls, so concurrent calls on unordered streams race."""
    _check(_lib.sar_fft_lines_static(n, n_lines, _ptr(inp), _ptr(out), 1 if inverse else 0, _stream(stream)))


def sar_transpose(rows: int, cols: int, inp, out, stream=None) -> None:
    _check(_lib.sar_transpose(rows, cols, _ptr(inp), _ptr(out), _stream(stream)))


def sar_plan_status(plan, stream=None) -> None:
    """Raise SarError(SAR_ERR_TIMEOUT) if a kernel of the plan gave up a bounded wait."""
    _check(_lib.sar_plan_status(_h(plan), _stream(stream)))


class Batch:
    """An opaque sar_batch handle."""

    def __init__(self, handle: int):
        self.handle = handle

    def destroy(self) -> None:
        if self.handle:
            _check(_lib.sar_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sar_batch_create(strips, flags: int = 0) -> Batch:
    """strips: sequence of dicts with n_range, n_az, raw, image,
    range_spectrum, az_spectrum (tensors or device addresses)."""
    arr = (sar_strip * len(strips))()
    for i, st in enumerate(strips):
        arr[i] = sar_strip(st["n_range"], st["n_az"], _ptr(st["raw"]), _ptr(st["image"]),
                           _ptr(st["range_spectrum"]), _ptr(st["az_spectrum"]))
    h = _vp()
    _check(_lib.sar_batch_create(arr, len(strips), flags, ctypes.byref(h)))
    return Batch(h.value)


def sar_batch_run(batch, stream=None) -> None:
    _check(_lib.sar_batch_run(_h(batch), _stream(stream)))


def sar_batch_status(batch, stream=None) -> None:
    """Raises SarError(SAR_ERR_TIMEOUT) if a bounded wait of the batch kernel
    ran out since the last call (the record is cleared)."""
    _check(_lib.sar_batch_status(_h(batch), _stream(stream)))


def sar_batch_info(batch) -> dict:
    info = sar_batch_info_t()
    _check(_lib.sar_batch_info(_h(batch), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def sar_batch_destroy(batch) -> None:
    batch.destroy()


class Server:
    """An opaque sar_server handle; keeps the config arrays alive."""

    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep

    def destroy(self) -> None:
        if self.handle:
            _check(_lib.sar_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def sar_server_create(classes, hbm_budget_bytes: int, max_inflight: int = 16, backfill_s: float = 0.05,
                      size_priority: bool = False, aging_s: float = 0.0) -> Server:
    """classes: sequence of dicts with n_range, n_az, pool, range_spectrum, az_spectrum."""
    k = len(classes)
    nr = (ctypes.c_int64 * k)(*[c["n_range"] for c in classes])
    na = (ctypes.c_int64 * k)(*[c["n_az"] for c in classes])
    pool = (ctypes.c_void_p * k)(*[_ptr(c["pool"]) for c in classes])
    hr = (ctypes.c_void_p * k)(*[_ptr(c["range_spectrum"]) for c in classes])
    ha = (ctypes.c_void_p * k)(*[_ptr(c["az_spectrum"]) for c in classes])
    cfg = sar_server_config(k, max_inflight, nr, na, pool, hr, ha, int(hbm_budget_bytes), float(backfill_s),
                            1 if size_priority else 0, float(aging_s))
    h = _vp()
    _check(_lib.sar_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return Server(h.value, (nr, na, pool, hr, ha, cfg, classes))


def sar_server_run(server, requests, mode: int = SAR_SERVE_OPEN_LOOP) -> list:
    """requests: sequence of (arrival_s, size_class[, output]); returns a list
    of dicts (arrival_s, admit_s, done_s, status, latency_s)."""
    n = len(requests)
    arr = (sar_request * max(1, n))()
    for i, r in enumerate(requests):
        arr[i] = sar_request(float(r[0]), int(r[1]), _ptr(r[2]) if len(r) > 2 and r[2] is not None else None)
    res = (sar_request_result * max(1, n))()
    _check(_lib.sar_server_run(_h(server), arr, n, mode, res))
    out = []
    for i in range(n):
        r = res[i]
        out.append(dict(arrival_s=r.arrival_s, admit_s=r.admit_s, done_s=r.done_s, status=r.status,
                        latency_s=r.done_s - r.arrival_s))
    return out


def sar_server_destroy(server) -> None:
    server.destroy()


def sar_sync(stream=None) -> None:
    _check(_lib.sar_sync(_stream(stream)))
