"""Thin ctypes binding of libsecpe.so (include/secpe.h): argument marshalling
only.  Every homomorphic step runs in the library's CUDA kernels; device
memory for ciphertexts comes from PyTorch tensors (uint64 words stored in
int64 tensors), streams are PyTorch's current CUDA stream.

The binding raises RuntimeError when the library is missing or a call
returns an error; there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsecpe.so")

# names exported by include/secpe.h
EXPORTS = [
    "secpe_ctx_create", "secpe_ctx_destroy", "secpe_ctx_primes", "secpe_ctx_n", "secpe_stream_status",
    "secpe_strerror", "secpe_keygen", "secpe_keys_destroy", "secpe_keys_export", "secpe_encrypt_coeffs",
    "secpe_encrypt", "secpe_encrypt_logits", "secpe_decrypt", "secpe_decrypt_coeffs", "secpe_ntt",
    "secpe_ntt_cts", "secpe_add", "secpe_sub", "secpe_mul_const", "secpe_add_const", "secpe_mul_relin",
    "secpe_rescale", "secpe_rotate", "secpe_keyswitch", "secpe_refresh_testonly", "secpe_sign", "secpe_max",
    "secpe_ensemble_aggregate", "secpe_encrypted_argmax", "secpe_argmax_batch", "secpe_argmax_batch_capture",
    "secpe_graph_launch", "secpe_graph_destroy", "secpe_get_counters",
    "secpe_reset_counters", "secpe_select_primes", "secpe_kprof_begin", "secpe_kprof_end", "secpe_kprof_report", "secpe_autotune",
    "secpe_tuning_set", "secpe_device_wait_selftest",
    "secpe_keyswitch_batch", "secpe_mul_relin_batch", "secpe_rotate_batch", "secpe_rescale_batch",
    "secpe_rescale_noalloc", "secpe_server_create", "secpe_server_destroy", "secpe_server_submit",
    "secpe_server_cancel", "secpe_server_step", "secpe_server_poll", "secpe_server_wait", "secpe_server_forget",
    "secpe_server_stats", "secpe_ntt_tc", "secpe_ntt_cts_tc", "secpe_expand_seeded", "secpe_keyswitch_batch_tc",
    "secpe_pool_usage", "secpe_mul32_probe", "secpe_packed_capacity", "secpe_encode_packed",
    "secpe_decode_packed", "secpe_encrypt_logits_packed", "secpe_decrypt_packed", "secpe_phoenix_argmax",
    "secpe_phoenix_argmax_batch", "secpe_linear_create", "secpe_linear_create_coeffs", "secpe_linear_destroy",
    "secpe_linear_apply", "secpe_encrypt_replicated", "secpe_boot_rotation_steps", "secpe_boot_create",
    "secpe_boot_create_coeffs", "secpe_boot_destroy", "secpe_bootstrap_batch", "secpe_bootstrap",
    "secpe_argmax_batch_boot", "secpe_level_plan", "secpe_ntt32_create", "secpe_ntt32_destroy", "secpe_ntt32",
    "secpe_bconv32", "secpe_rotate_hoisted", "secpe_keyswitch32",
]


class ParamsC(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in (
        "log_n", "q0_bits", "q_bits", "n_q", "p_bits", "n_p", "dnum", "log_scale", "sign_dg", "sign_df",
        "reserve", "secret_hw", "boot_primes", "boot_bits")]


class CtC(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("level", ctypes.c_int32), ("cap", ctypes.c_int32),
                ("scale", ctypes.c_double)]


class QueryC(ctypes.Structure):
    _fields_ = [("cts", ctypes.POINTER(CtC)), ("K", ctypes.c_int32), ("C", ctypes.c_int32),
                ("d_min", ctypes.c_double), ("d_max", ctypes.c_double), ("qseed", ctypes.c_uint64),
                ("z_out", ctypes.POINTER(CtC)), ("keys", ctypes.c_void_p)]


class CtBatchC(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("batch", ctypes.c_int32), ("cap", ctypes.c_int32),
                ("level", ctypes.c_int32), ("scale", ctypes.c_double), ("stride", ctypes.c_uint64)]


class ServerStatsC(ctypes.Structure):
    _fields_ = [("waiting", ctypes.c_int32), ("active", ctypes.c_int32), ("done", ctypes.c_int32),
                ("in_flight_bytes", ctypes.c_uint64), ("keys_bytes", ctypes.c_uint64),
                ("scratch_bytes", ctypes.c_uint64)]


class CountersC(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "rotations", "signs", "relins", "refreshes", "keyswitches", "launches", "bootstraps")]


class TuningC(ctypes.Structure):
    _fields_ = [("n_kernels", ctypes.c_int32), ("name", (ctypes.c_char * 32) * 8),
                ("ctas_per_sm", ctypes.c_int32 * 8), ("ms", (ctypes.c_float * 2) * 8)]


class KprofC(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("model_bytes", ctypes.c_double), ("mul32", ctypes.c_double)]


_lib = None


def lib():
    """Load libsecpe.so (built by paper_2502_00847_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsecpe.so is not built (run paper_2502_00847_gb300.build.build()): %s" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "secpe_ctx_create": (i32, [P(ParamsC), P(vp)]),
        "secpe_ctx_destroy": (None, [vp]),
        "secpe_ctx_primes": (i32, [vp, P(u64)]),
        "secpe_ctx_n": (i32, [vp]),
        "secpe_stream_status": (i32, [vp, vp, P(i32)]),
        "secpe_strerror": (ctypes.c_char_p, [i32]),
        "secpe_keygen": (i32, [vp, u64, P(i32), i32, P(vp)]),
        "secpe_keys_destroy": (None, [vp]),
        "secpe_keys_export": (i32, [vp, vp, i32, i32, P(u64), ctypes.c_size_t]),
        "secpe_encrypt_coeffs": (i32, [vp, vp, P(ctypes.c_int64), i32, dbl, u64, P(CtC), vp]),
        "secpe_encrypt": (i32, [vp, vp, P(dbl), i32, u64, P(CtC), vp]),
        "secpe_encrypt_logits": (i32, [vp, vp, P(dbl), i32, dbl, u64, P(CtC), vp]),
        "secpe_decrypt": (i32, [vp, vp, P(CtC), P(dbl), i32, vp]),
        "secpe_decrypt_coeffs": (i32, [vp, vp, P(CtC), P(dbl), vp]),
        "secpe_ntt": (i32, [vp, vp, P(i32), i32, i32, vp]),
        "secpe_ntt_cts": (i32, [vp, vp, i32, ctypes.c_size_t, i32, i32, i32, vp]),
        "secpe_add": (i32, [vp, P(CtC), P(CtC), P(CtC), vp]),
        "secpe_sub": (i32, [vp, P(CtC), P(CtC), P(CtC), vp]),
        "secpe_mul_const": (i32, [vp, P(CtC), dbl, dbl, i32, P(CtC), vp]),
        "secpe_add_const": (i32, [vp, P(CtC), dbl, P(CtC), vp]),
        "secpe_mul_relin": (i32, [vp, vp, P(CtC), P(CtC), P(CtC), vp]),
        "secpe_rescale": (i32, [vp, P(CtC), P(CtC), vp]),
        "secpe_rotate": (i32, [vp, vp, P(CtC), i32, P(CtC), vp]),
        "secpe_keyswitch": (i32, [vp, vp, i32, vp, i32, i32, vp, vp, vp]),
        "secpe_refresh_testonly": (i32, [vp, vp, P(CtC), u64, u64, P(CtC), vp]),
        "secpe_sign": (i32, [vp, vp, P(CtC), i32, u64, P(u64), P(CtC), vp]),
        "secpe_max": (i32, [vp, vp, P(CtC), P(CtC), u64, P(u64), P(CtC), vp]),
        "secpe_ensemble_aggregate": (i32, [vp, P(CtC), i32, dbl, dbl, P(CtC), vp]),
        "secpe_encrypted_argmax": (i32, [vp, vp, P(CtC), i32, u64, P(CtC), vp]),
        "secpe_argmax_batch": (i32, [vp, vp, P(QueryC), i32, vp]),
        "secpe_argmax_batch_capture": (i32, [vp, vp, P(QueryC), i32, P(vp), P(ctypes.c_int64)]),
        "secpe_graph_launch": (i32, [vp, vp]),
        "secpe_graph_destroy": (None, [vp]),
        "secpe_get_counters": (i32, [vp, P(CountersC)]),
        "secpe_reset_counters": (i32, [vp]),
        "secpe_select_primes": (i32, [P(ParamsC), P(u64), i32]),
        "secpe_kprof_begin": (i32, [vp, ctypes.c_char_p, i32]),
        "secpe_kprof_end": (i32, [vp, P(KprofC)]),
        "secpe_kprof_report": (i32, [vp, ctypes.c_char_p, ctypes.c_size_t, P(ctypes.c_size_t)]),
        "secpe_autotune": (i32, [vp, P(TuningC), vp]),
        "secpe_tuning_set": (i32, [vp, i32, i32]),
        "secpe_device_wait_selftest": (i32, [vp, i32, ctypes.c_int64, vp]),
        "secpe_keyswitch_batch": (i32, [vp, vp, i32, P(CtBatchC), P(CtBatchC), vp]),
        "secpe_keyswitch_batch_tc": (i32, [vp, vp, i32, P(CtBatchC), P(CtBatchC), vp]),
        "secpe_mul_relin_batch": (i32, [vp, vp, P(CtBatchC), P(CtBatchC), P(CtBatchC), vp]),
        "secpe_rotate_batch": (i32, [vp, vp, P(CtBatchC), i32, P(CtBatchC), vp]),
        "secpe_rescale_batch": (i32, [vp, P(CtBatchC), P(CtBatchC), vp]),
        "secpe_rescale_noalloc": (i32, [vp, P(CtC), P(CtC), vp]),
        "secpe_server_create": (i32, [vp, vp, u64, i32, P(vp)]),
        "secpe_server_destroy": (None, [vp]),
        "secpe_server_submit": (i32, [vp, P(QueryC), P(ctypes.c_int64)]),
        "secpe_server_cancel": (i32, [vp, ctypes.c_int64]),
        "secpe_server_step": (i32, [vp, vp, P(i32)]),
        "secpe_server_poll": (i32, [vp, ctypes.c_int64, P(i32)]),
        "secpe_server_wait": (i32, [vp, ctypes.c_int64, dbl]),
        "secpe_server_forget": (i32, [vp, ctypes.c_int64]),
        "secpe_server_stats": (i32, [vp, P(ServerStatsC)]),
        "secpe_ntt_tc": (i32, [vp, vp, P(i32), i32, i32, vp]),
        "secpe_ntt_cts_tc": (i32, [vp, vp, i32, ctypes.c_size_t, i32, i32, i32, vp]),
        "secpe_expand_seeded": (i32, [vp, vp, i32, ctypes.c_size_t, i32, i32, P(u64), vp]),
        "secpe_pool_usage": (i32, [i32, P(u64), P(u64)]),
        "secpe_mul32_probe": (i32, [vp, i32, i32, P(dbl), vp]),
        "secpe_packed_capacity": (i32, [i32, i32]),
        "secpe_phoenix_argmax": (i32, [vp, vp, P(CtC), i32, u64, P(CtC), vp]),
        "secpe_phoenix_argmax_batch": (i32, [vp, vp, P(QueryC), i32, vp]),
        "secpe_linear_create": (i32, [vp, P(dbl), i32, i32, i32, dbl, P(vp)]),
        "secpe_linear_create_coeffs": (i32, [vp, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int64), i32, i32,
                                             i32, P(vp)]),
        "secpe_linear_destroy": (None, [vp]),
        "secpe_linear_apply": (i32, [vp, vp, vp, P(CtC), P(CtC), vp]),
        "secpe_encrypt_replicated": (i32, [vp, vp, P(dbl), i32, i32, u64, P(CtC), vp]),
        "secpe_boot_rotation_steps": (i32, [vp, i32, P(i32), i32, P(i32)]),
        "secpe_level_plan": (i32, [P(ParamsC), i32, i32, i32, P(i32), i32, P(i32)]),
        "secpe_ntt32_create": (i32, [i32, P(ctypes.c_uint32), i32, P(vp)]),
        "secpe_ntt32_destroy": (None, [vp]),
        "secpe_ntt32": (i32, [vp, vp, P(i32), i32, i32, vp]),
        "secpe_bconv32": (i32, [vp, vp, P(i32), i32, vp, P(i32), i32, i32, vp]),
        "secpe_rotate_hoisted": (i32, [vp, vp, P(CtC), P(i32), i32, P(CtC), vp]),
        "secpe_keyswitch32": (i32, [vp, vp, P(i32), i32, P(i32), i32, i32, vp, vp, i32, i32, vp]),
        "secpe_boot_create": (i32, [vp, i32, P(vp)]),
        "secpe_boot_create_coeffs": (i32, [vp, i32, P(ctypes.c_int64), P(ctypes.c_int64), P(vp)]),
        "secpe_boot_destroy": (None, [vp]),
        "secpe_bootstrap_batch": (i32, [vp, vp, vp, P(CtBatchC), P(CtBatchC), vp]),
        "secpe_bootstrap": (i32, [vp, vp, vp, P(CtC), P(CtC), vp]),
        "secpe_argmax_batch_boot": (i32, [vp, vp, vp, P(QueryC), i32, vp]),
        "secpe_encode_packed": (i32, [i32, dbl, P(dbl), i32, i32, dbl, P(ctypes.c_int64)]),
        "secpe_decode_packed": (i32, [i32, dbl, P(dbl), i32, i32, P(dbl)]),
        "secpe_encrypt_logits_packed": (i32, [vp, vp, P(dbl), i32, i32, dbl, u64, P(CtC), vp]),
        "secpe_decrypt_packed": (i32, [vp, vp, P(CtC), i32, i32, P(dbl), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def select_primes(**params):
    """Host-only prime selection (no GPU needed): (ciphertext primes, special)."""
    p = ParamsC(**{f[0]: params.get(f[0], 0) for f in ParamsC._fields_})
    out = np.zeros(p.n_q + p.n_p, dtype=np.uint64)
    _check(lib().secpe_select_primes(ctypes.byref(p), _u64p(out), len(out)), "secpe_select_primes")
    vals = [int(x) for x in out]
    return vals[: p.n_q], vals[p.n_q:]


def level_plan(C, entry_level, refresh_level, **params):
    """Host-only secpe_level_plan: the levels of y entering round 0 and right
    after each refresh of Alg. 1 (level-aware QuickMax)."""
    p = ParamsC(**{f[0]: params.get(f[0], 0) for f in ParamsC._fields_})
    cnt = ctypes.c_int32(0)
    _check(lib().secpe_level_plan(ctypes.byref(p), C, entry_level, refresh_level, None, 0, ctypes.byref(cnt)),
           "secpe_level_plan")
    arr = (ctypes.c_int32 * cnt.value)()
    _check(lib().secpe_level_plan(ctypes.byref(p), C, entry_level, refresh_level, arr, cnt.value, ctypes.byref(cnt)),
           "secpe_level_plan")
    return list(arr)


class SecpeError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().secpe_strerror(code).decode()
        super().__init__("%s failed: %s (%d)" % (where, msg, code))
        self.code = code


STEP_CONJ = 0x40000000  # SECPE_STEP_CONJ: the conjugation "rotation"


def _check(code, where):
    if code != 0:
        raise SecpeError(code, where)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _u64p(arr):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


class Context:
    """secpe_ctx: primes, NTT and base-conversion tables on the device."""

    def __init__(self, log_n, q0_bits, q_bits, n_q, p_bits, n_p, dnum, log_scale, sign_dg=2, sign_df=2,
                 reserve=1, secret_hw=0, boot_primes=0, boot_bits=0):
        self.params = dict(log_n=log_n, q0_bits=q0_bits, q_bits=q_bits, n_q=n_q, p_bits=p_bits, n_p=n_p,
                           dnum=dnum, log_scale=log_scale, sign_dg=sign_dg, sign_df=sign_df, reserve=reserve,
                           secret_hw=secret_hw, boot_primes=boot_primes, boot_bits=boot_bits)
        p = ParamsC(**self.params)
        h = ctypes.c_void_p()
        _check(lib().secpe_ctx_create(ctypes.byref(p), ctypes.byref(h)), "secpe_ctx_create")
        self.h = h
        self.n = 1 << log_n
        self.n_q, self.n_p = n_q, n_p
        self.L = n_q - 1
        self.scale = float(2 ** log_scale)

    @classmethod
    def from_params(cls, p):
        """From any object with the secpe_params field names as attributes."""
        return cls(**{f[0]: getattr(p, f[0]) for f in ParamsC._fields_})

    def primes(self):
        out = np.zeros(self.n_q + self.n_p, dtype=np.uint64)
        _check(lib().secpe_ctx_primes(self.h, _u64p(out)), "secpe_ctx_primes")
        return [int(x) for x in out]

    def close(self):
        if self.h:
            lib().secpe_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def counters(self):
        c = CountersC()
        _check(lib().secpe_get_counters(self.h, ctypes.byref(c)), "secpe_get_counters")
        return {f[0]: int(getattr(c, f[0])) for f in CountersC._fields_}

    def reset_counters(self):
        _check(lib().secpe_reset_counters(self.h), "secpe_reset_counters")

    def kprof_begin(self, name_filter, max_launches=200000):
        _check(lib().secpe_kprof_begin(self.h, name_filter.encode(), max_launches), "secpe_kprof_begin")

    def kprof_end(self):
        k = KprofC()
        _check(lib().secpe_kprof_end(self.h, ctypes.byref(k)), "secpe_kprof_end")
        return dict(launches=int(k.launches), total_ms=float(k.total_ms), bytes=float(k.bytes),
                    model_bytes=float(k.model_bytes), mul32=float(k.mul32))

    def mul32_probe(self, ctas_per_sm=8, iters=4096):
        """secpe_mul32_probe: achieved 32-bit multiplies per second of the
        128-bit multiply-accumulate form on this GPU."""
        r = ctypes.c_double(0.0)
        _check(lib().secpe_mul32_probe(self.h, ctas_per_sm, iters, ctypes.byref(r), _stream()), "secpe_mul32_probe")
        return float(r.value)

    def autotune(self):
        """Times the candidate launch configurations of the N = 2^16 kernels and
        keeps the fastest; returns {kernel: {"ctas_per_sm", "ms_3", "ms_4"}}."""
        t = TuningC()
        _check(lib().secpe_autotune(self.h, ctypes.byref(t), _stream()), "secpe_autotune")
        return {t.name[i].value.decode(): {"ctas_per_sm": int(t.ctas_per_sm[i]), "ms_3": float(t.ms[i][0]),
                                           "ms_4": float(t.ms[i][1])} for i in range(t.n_kernels)}

    def tuning_set(self, kernel, ctas_per_sm):
        _check(lib().secpe_tuning_set(self.h, kernel, ctas_per_sm), "secpe_tuning_set")

    def kprof_report(self):
        """Per-kernel (name, launches, ms) of the last kprof_begin("*") .. kprof_end range."""
        need = ctypes.c_size_t()
        _check(lib().secpe_kprof_report(self.h, None, 0, ctypes.byref(need)), "secpe_kprof_report")
        buf = ctypes.create_string_buffer(need.value)
        _check(lib().secpe_kprof_report(self.h, buf, need.value, ctypes.byref(need)), "secpe_kprof_report")
        rows = []
        for line in buf.value.decode().splitlines():
            name, n, ms = line.split("\t")
            rows.append((name, int(n), float(ms)))
        return rows

    def device_wait_selftest(self, arrive, polls=1 << 16):
        _check(lib().secpe_device_wait_selftest(self.h, 1 if arrive else 0, polls, _stream()),
               "secpe_device_wait_selftest")

    def stream_status(self):
        v = ctypes.c_int32()
        _check(lib().secpe_stream_status(self.h, _stream(), ctypes.byref(v)), "secpe_stream_status")
        return int(v.value)

    # ---------------------------------------------------------------- data
    def new_ct(self, cap=None, device="cuda"):
        """A zeroed ciphertext buffer [2][cap][N] (int64 storage of uint64)."""
        import torch
        cap = self.L + 1 if cap is None else cap
        return Ciphertext(torch.zeros((2, cap, self.n), dtype=torch.int64, device=device), 0, self.scale)


class Ciphertext:
    """A device ciphertext: tensor [2][cap][N] plus level and scale."""

    def __init__(self, data, level, scale):
        self.data = data
        self.level = level
        self.scale = scale

    @property
    def cap(self):
        return int(self.data.shape[1])

    def struct(self):
        return CtC(ctypes.c_void_p(self.data.data_ptr()), self.level, self.cap, self.scale)

    def update(self, c):
        self.level = int(c.level)
        self.scale = float(c.scale)

    def residues(self):
        """Limbs 0..level of both polynomials as a numpy uint64 array."""
        return self.data[:, : self.level + 1].cpu().numpy().view(np.uint64)

    @staticmethod
    def from_residues(arr, level, scale, cap=None):
        import torch
        arr = np.ascontiguousarray(arr, dtype=np.uint64)
        cap = arr.shape[1] if cap is None else cap
        t = torch.zeros((2, cap, arr.shape[2]), dtype=torch.int64)
        t[:, : arr.shape[1]] = torch.from_numpy(arr.view(np.int64))
        return Ciphertext(t.cuda(), level, scale)


class Keys:
    def __init__(self, ctx, seed, rot_steps=()):
        steps = (ctypes.c_int32 * max(1, len(rot_steps)))(*rot_steps)
        h = ctypes.c_void_p()
        _check(lib().secpe_keygen(ctx.h, ctypes.c_uint64(seed), steps, len(rot_steps), ctypes.byref(h)),
               "secpe_keygen")
        self.h = h
        self.ctx = ctx

    def close(self):
        if self.h:
            lib().secpe_keys_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self, which, step=0):
        n = self.ctx.n
        npr = self.ctx.n_q + self.ctx.n_p
        alpha = -(-self.ctx.n_q // self.ctx.params["dnum"])
        ndig = -(-self.ctx.n_q // alpha)
        words = npr * n if which == 0 else ndig * 2 * npr * n
        out = np.zeros(words, dtype=np.uint64)
        _check(lib().secpe_keys_export(self.ctx.h, self.h, which, step, _u64p(out), words), "secpe_keys_export")
        return out.reshape((npr, n) if which == 0 else (ndig, 2, npr, n))


# ------------------------------------------------------------------ client
def encrypt_coeffs(ctx, keys, m, level, scale, seed, out=None):
    m = np.ascontiguousarray(m, dtype=np.int64)
    out = ctx.new_ct() if out is None else out
    c = out.struct()
    _check(lib().secpe_encrypt_coeffs(ctx.h, keys.h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), level,
                                      scale, ctypes.c_uint64(seed), ctypes.byref(c), _stream()),
           "secpe_encrypt_coeffs")
    out.update(c)
    return out


def encrypt(ctx, keys, v, seed, out=None):
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = ctx.new_ct() if out is None else out
    c = out.struct()
    _check(lib().secpe_encrypt(ctx.h, keys.h, v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(v),
                               ctypes.c_uint64(seed), ctypes.byref(c), _stream()), "secpe_encrypt")
    out.update(c)
    return out


def encrypt_logits(ctx, keys, v, d_min, seed, out=None):
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = ctx.new_ct() if out is None else out
    c = out.struct()
    _check(lib().secpe_encrypt_logits(ctx.h, keys.h, v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(v),
                                      d_min, ctypes.c_uint64(seed), ctypes.byref(c), _stream()),
           "secpe_encrypt_logits")
    out.update(c)
    return out


def _dblp(arr):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def packed_capacity(log_n, C):
    """secpe_packed_capacity: inputs of C classes per ciphertext."""
    r = lib().secpe_packed_capacity(log_n, C)
    if r < 0:
        raise SecpeError(r, "secpe_packed_capacity")
    return r


def encode_packed(log_n, scale, v, d_min):
    """secpe_encode_packed (host only): coefficients of the packed slot vector of v[P][C]."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    P, C = v.shape
    m = np.zeros(1 << log_n, dtype=np.int64)
    _check(lib().secpe_encode_packed(log_n, scale, _dblp(v), P, C, d_min,
                                     m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "secpe_encode_packed")
    return m


def decode_packed(log_n, scale, coeffs, P, C):
    """secpe_decode_packed (host only): out[P][C] from centred coefficients."""
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64)
    out = np.zeros((P, C), dtype=np.float64)
    _check(lib().secpe_decode_packed(log_n, scale, _dblp(coeffs), P, C, _dblp(out)), "secpe_decode_packed")
    return out


def encrypt_logits_packed(ctx, keys, v, d_min, seed, out=None):
    """secpe_encrypt_logits_packed: one prompt's logits of P inputs, v[P][C]."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    P, C = v.shape
    out = ctx.new_ct() if out is None else out
    c = out.struct()
    _check(lib().secpe_encrypt_logits_packed(ctx.h, keys.h, _dblp(v), P, C, d_min, ctypes.c_uint64(seed),
                                             ctypes.byref(c), _stream()), "secpe_encrypt_logits_packed")
    out.update(c)
    return out


def decrypt_packed(ctx, keys, ct, P, C):
    """secpe_decrypt_packed: out[P][C], the first C slots of every block."""
    out = np.zeros((P, C), dtype=np.float64)
    c = ct.struct()
    _check(lib().secpe_decrypt_packed(ctx.h, keys.h, ctypes.byref(c), P, C, _dblp(out), _stream()),
           "secpe_decrypt_packed")
    return out


def expand_seeded(ctx, cts_tensor, level, seeds):
    """Regenerate c1 of `cts_tensor` ([batch][2][cap][N]) from the encryption seeds."""
    seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
    batch, cap, n = int(cts_tensor.shape[0]), int(cts_tensor.shape[2]), int(cts_tensor.shape[3])
    _check(lib().secpe_expand_seeded(ctx.h, ctypes.c_void_p(cts_tensor.data_ptr()), batch, 2 * cap * n, cap, level,
                                     _u64p(seeds), _stream()), "secpe_expand_seeded")


def decrypt(ctx, keys, ct, n):
    out = np.zeros(n, dtype=np.float64)
    c = ct.struct()
    _check(lib().secpe_decrypt(ctx.h, keys.h, ctypes.byref(c), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               n, _stream()), "secpe_decrypt")
    return out


def decrypt_coeffs(ctx, keys, ct):
    out = np.zeros(ctx.n, dtype=np.float64)
    c = ct.struct()
    _check(lib().secpe_decrypt_coeffs(ctx.h, keys.h, ctypes.byref(c),
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream()),
           "secpe_decrypt_coeffs")
    return out


# -------------------------------------------------------------- primitives
def ntt(ctx, limbs, prime_idx, inverse=False):
    """In-place (I)NTT of a [count][N] int64 CUDA tensor of residues."""
    pi = (ctypes.c_int32 * len(prime_idx))(*prime_idx)
    _check(lib().secpe_ntt(ctx.h, ctypes.c_void_p(limbs.data_ptr()), pi, len(prime_idx), 1 if inverse else 0,
                           _stream()), "secpe_ntt")
    return limbs


def ntt_tc(ctx, limbs, prime_idx, inverse=False):
    """Precision variant of ntt(): column pass on the tensor pipe (N = 2^16)."""
    pi = (ctypes.c_int32 * len(prime_idx))(*prime_idx)
    _check(lib().secpe_ntt_tc(ctx.h, ctypes.c_void_p(limbs.data_ptr()), pi, len(prime_idx), 1 if inverse else 0,
                              _stream()), "secpe_ntt_tc")
    return limbs


def ntt_cts_tc(ctx, base, batch, ct_stride, cap, level, inverse=False):
    _check(lib().secpe_ntt_cts_tc(ctx.h, ctypes.c_void_p(base.data_ptr()), batch, ct_stride, cap, level,
                                  1 if inverse else 0, _stream()), "secpe_ntt_cts_tc")


def ntt_cts(ctx, base, batch, ct_stride, cap, level, inverse=False):
    _check(lib().secpe_ntt_cts(ctx.h, ctypes.c_void_p(base.data_ptr()), batch, ct_stride, cap, level,
                               1 if inverse else 0, _stream()), "secpe_ntt_cts")


def _binary(fn, name, ctx, a, b, out=None):
    out = ctx.new_ct() if out is None else out
    ca, cb, co = a.struct(), b.struct(), out.struct()
    _check(fn(ctx.h, ctypes.byref(ca), ctypes.byref(cb), ctypes.byref(co), _stream()), name)
    out.update(co)
    return out


def add(ctx, a, b, out=None):
    return _binary(lib().secpe_add, "secpe_add", ctx, a, b, out)


def sub(ctx, a, b, out=None):
    return _binary(lib().secpe_sub, "secpe_sub", ctx, a, b, out)


def mul_const(ctx, a, c, target_scale, out_level, out=None):
    out = ctx.new_ct() if out is None else out
    ca, co = a.struct(), out.struct()
    _check(lib().secpe_mul_const(ctx.h, ctypes.byref(ca), c, target_scale, out_level, ctypes.byref(co), _stream()),
           "secpe_mul_const")
    out.update(co)
    return out


def add_const(ctx, a, c, out=None):
    out = ctx.new_ct() if out is None else out
    ca, co = a.struct(), out.struct()
    _check(lib().secpe_add_const(ctx.h, ctypes.byref(ca), c, ctypes.byref(co), _stream()), "secpe_add_const")
    out.update(co)
    return out


def mul_relin(ctx, keys, a, b, out=None):
    out = ctx.new_ct() if out is None else out
    ca, cb, co = a.struct(), b.struct(), out.struct()
    _check(lib().secpe_mul_relin(ctx.h, keys.h, ctypes.byref(ca), ctypes.byref(cb), ctypes.byref(co), _stream()),
           "secpe_mul_relin")
    out.update(co)
    return out


def rescale(ctx, a, out=None):
    out = ctx.new_ct() if out is None else out
    ca, co = a.struct(), out.struct()
    _check(lib().secpe_rescale(ctx.h, ctypes.byref(ca), ctypes.byref(co), _stream()), "secpe_rescale")
    out.update(co)
    return out


def rescale_noalloc(ctx, a, out):
    """secpe_rescale_noalloc: the rescale with no device allocation (scratch is
    a fixed array inside the library); `out` must be preallocated."""
    ca, co = a.struct(), out.struct()
    _check(lib().secpe_rescale_noalloc(ctx.h, ctypes.byref(ca), ctypes.byref(co), _stream()),
           "secpe_rescale_noalloc")
    out.update(co)
    return out


def pool_usage(trim=False):
    """secpe_pool_usage: (used, reserved) bytes of the current device's
    stream-ordered pool, after returning its unused blocks when trim."""
    used, reserved = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().secpe_pool_usage(1 if trim else 0, ctypes.byref(used), ctypes.byref(reserved)), "secpe_pool_usage")
    return int(used.value), int(reserved.value)


def rotate(ctx, keys, a, steps, out=None):
    out = ctx.new_ct() if out is None else out
    ca, co = a.struct(), out.struct()
    _check(lib().secpe_rotate(ctx.h, keys.h, ctypes.byref(ca), steps, ctypes.byref(co), _stream()), "secpe_rotate")
    out.update(co)
    return out


def rotate_hoisted(ctx, keys, a, steps, outs=None):
    """secpe_rotate_hoisted: rotations of a by every step from one ModUp."""
    outs = [ctx.new_ct() for _ in steps] if outs is None else outs
    ca = a.struct()
    arr = (CtC * len(steps))(*[o.struct() for o in outs])
    st = (ctypes.c_int32 * len(steps))(*steps)
    _check(lib().secpe_rotate_hoisted(ctx.h, keys.h, ctypes.byref(ca), st, len(steps), arr, _stream()),
           "secpe_rotate_hoisted")
    for o, c in zip(outs, arr):
        o.update(c)
    return outs


def keyswitch(ctx, keys, galois_step, d, level):
    """Key switching of one polynomial d (tensor [cap][N]); returns (ks0, ks1)."""
    import torch
    cap = int(d.shape[0])
    ks0 = torch.zeros((cap, ctx.n), dtype=torch.int64, device=d.device)
    ks1 = torch.zeros_like(ks0)
    _check(lib().secpe_keyswitch(ctx.h, keys.h, galois_step, ctypes.c_void_p(d.data_ptr()), level, cap,
                                 ctypes.c_void_p(ks0.data_ptr()), ctypes.c_void_p(ks1.data_ptr()), _stream()),
           "secpe_keyswitch")
    return ks0, ks1


def refresh_testonly(ctx, keys, a, qseed, refresh_index, out=None):
    out = ctx.new_ct() if out is None else out
    ca, co = a.struct(), out.struct()
    _check(lib().secpe_refresh_testonly(ctx.h, keys.h, ctypes.byref(ca), ctypes.c_uint64(qseed),
                                        ctypes.c_uint64(refresh_index), ctypes.byref(co), _stream()),
           "secpe_refresh_testonly")
    out.update(co)
    return out


def sign(ctx, keys, x, out_levels, qseed, refresh_index=0, out=None):
    out = ctx.new_ct() if out is None else out
    cx, co = x.struct(), out.struct()
    ri = ctypes.c_uint64(refresh_index)
    _check(lib().secpe_sign(ctx.h, keys.h, ctypes.byref(cx), out_levels, ctypes.c_uint64(qseed), ctypes.byref(ri),
                            ctypes.byref(co), _stream()), "secpe_sign")
    out.update(co)
    return out, int(ri.value)


def vmax(ctx, keys, a, y, qseed, refresh_index=0, out=None):
    out = ctx.new_ct() if out is None else out
    ca, cy, co = a.struct(), y.struct(), out.struct()
    ri = ctypes.c_uint64(refresh_index)
    _check(lib().secpe_max(ctx.h, keys.h, ctypes.byref(ca), ctypes.byref(cy), ctypes.c_uint64(qseed),
                           ctypes.byref(ri), ctypes.byref(co), _stream()), "secpe_max")
    out.update(co)
    return out, int(ri.value)


def ensemble_aggregate(ctx, cts, d_min, d_max, out=None):
    out = ctx.new_ct() if out is None else out
    arr = (CtC * len(cts))(*[c.struct() for c in cts])
    co = out.struct()
    _check(lib().secpe_ensemble_aggregate(ctx.h, arr, len(cts), d_min, d_max, ctypes.byref(co), _stream()),
           "secpe_ensemble_aggregate")
    out.update(co)
    return out


def encrypted_argmax(ctx, keys, y, C, qseed, out=None):
    out = ctx.new_ct() if out is None else out
    cy, co = y.struct(), out.struct()
    _check(lib().secpe_encrypted_argmax(ctx.h, keys.h, ctypes.byref(cy), C, ctypes.c_uint64(qseed),
                                        ctypes.byref(co), _stream()), "secpe_encrypted_argmax")
    out.update(co)
    return out


def _query_array(queries):
    keep = []
    qarr = (QueryC * len(queries))()
    for i, q in enumerate(queries):
        cts = (CtC * len(q["cts"]))(*[c.struct() for c in q["cts"]])
        z = q["z_out"].struct()
        keep.append((cts, z))
        tk = q.get("keys")
        qarr[i] = QueryC(cts, len(q["cts"]), q["C"], q["d_min"], q["d_max"], q["qseed"], ctypes.pointer(z),
                         tk.h.value if tk is not None else None)
    return qarr, keep


def argmax_batch(ctx, keys, queries):
    """queries: list of dicts with cts (list of Ciphertext), C, d_min, d_max,
    qseed, z_out (Ciphertext).  Updates each z_out's level/scale."""
    qarr, keep = _query_array(queries)
    _check(lib().secpe_argmax_batch(ctx.h, keys.h, qarr, len(queries), _stream()), "secpe_argmax_batch")
    for q, (_, z) in zip(queries, keep):
        q["z_out"].update(z)


def phoenix_argmax(ctx, keys, y, C, qseed, out=None):
    """secpe_phoenix_argmax: the Phoenix baseline Argmax on a normalised y."""
    out = ctx.new_ct() if out is None else out
    cy, co = y.struct(), out.struct()
    _check(lib().secpe_phoenix_argmax(ctx.h, keys.h, ctypes.byref(cy), C, ctypes.c_uint64(qseed),
                                      ctypes.byref(co), _stream()), "secpe_phoenix_argmax")
    out.update(co)
    return out


def phoenix_argmax_batch(ctx, keys, queries):
    """secpe_phoenix_argmax_batch: aggregation + Phoenix Argmax, batched
    (queries as for argmax_batch)."""
    qarr, keep = _query_array(queries)
    _check(lib().secpe_phoenix_argmax_batch(ctx.h, keys.h, qarr, len(queries), _stream()),
           "secpe_phoenix_argmax_batch")
    for q, (_, z) in zip(queries, keep):
        q["z_out"].update(z)


def encrypt_replicated(ctx, keys, x, C, seed, out=None):
    """secpe_encrypt_replicated: x[d] with x[j] in the C' slots [j C', (j+1) C')."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = ctx.new_ct() if out is None else out
    c = out.struct()
    _check(lib().secpe_encrypt_replicated(ctx.h, keys.h, _dblp(x), len(x), C, ctypes.c_uint64(seed),
                                          ctypes.byref(c), _stream()), "secpe_encrypt_replicated")
    out.update(c)
    return out


class Linear:
    """secpe_linear: the encoded plaintext weights of the CLIP-style linear
    step (from T[K][C][d] doubles, or from integer coefficients)."""

    def __init__(self, ctx, T=None, d_min=None, coeffs=None, K=None, C=None, d=None):
        h = ctypes.c_void_p()
        if coeffs is None:
            T = np.ascontiguousarray(T, dtype=np.float64)
            K, C, d = T.shape
            _check(lib().secpe_linear_create(ctx.h, _dblp(T), K, C, d, d_min, ctypes.byref(h)), "secpe_linear_create")
        else:
            Wm, mask, pad = (np.ascontiguousarray(np.asarray(a, dtype=np.int64)) for a in coeffs)
            i64p = ctypes.POINTER(ctypes.c_int64)
            _check(lib().secpe_linear_create_coeffs(ctx.h, Wm.ctypes.data_as(i64p), mask.ctypes.data_as(i64p),
                                                    pad.ctypes.data_as(i64p), K, C, d, ctypes.byref(h)),
                   "secpe_linear_create_coeffs")
        self.h, self.ctx, self.K = h, ctx, K

    def apply(self, keys, x, outs=None):
        """The K logit ciphertexts of x (secpe_linear_apply)."""
        outs = [self.ctx.new_ct() for _ in range(self.K)] if outs is None else outs
        arr = (CtC * self.K)(*[o.struct() for o in outs])
        cx = x.struct()
        _check(lib().secpe_linear_apply(self.ctx.h, keys.h, self.h, ctypes.byref(cx), arr, _stream()),
               "secpe_linear_apply")
        for o, c in zip(outs, arr):
            o.update(c)
        return outs

    def close(self):
        if self.h:
            lib().secpe_linear_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def boot_rotation_steps(ctx, n):
    """secpe_boot_rotation_steps: the Galois key steps bootstrapping needs."""
    cnt = ctypes.c_int32(0)
    _check(lib().secpe_boot_rotation_steps(ctx.h, n, None, 0, ctypes.byref(cnt)), "secpe_boot_rotation_steps")
    arr = (ctypes.c_int32 * cnt.value)()
    _check(lib().secpe_boot_rotation_steps(ctx.h, n, arr, cnt.value, ctypes.byref(cnt)), "secpe_boot_rotation_steps")
    return list(arr)


class Boot:
    """secpe_boot: a bootstrapping plan for blocks of n slots (plaintext
    diagonals from the library's encoder, or from integer coefficients)."""

    def __init__(self, ctx, n, coeffs=None):
        h = ctypes.c_void_p()
        if coeffs is None:
            _check(lib().secpe_boot_create(ctx.h, n, ctypes.byref(h)), "secpe_boot_create")
        else:
            c2s, s2c = (np.ascontiguousarray(np.asarray(a, dtype=np.int64)) for a in coeffs)
            i64p = ctypes.POINTER(ctypes.c_int64)
            _check(lib().secpe_boot_create_coeffs(ctx.h, n, c2s.ctypes.data_as(i64p), s2c.ctypes.data_as(i64p),
                                                  ctypes.byref(h)), "secpe_boot_create_coeffs")
        self.h, self.ctx, self.n = h, ctx, n

    def bootstrap(self, keys, ct, out=None):
        out = self.ctx.new_ct() if out is None else out
        ci, co = ct.struct(), out.struct()
        _check(lib().secpe_bootstrap(self.ctx.h, keys.h, self.h, ctypes.byref(ci), ctypes.byref(co), _stream()),
               "secpe_bootstrap")
        out.update(co)
        return out

    def bootstrap_batch(self, keys, a, out):
        """a, out: CtBatch (out's level/scale are set)."""
        ca, co = a.struct(), out.struct()
        _check(lib().secpe_bootstrap_batch(self.ctx.h, keys.h, self.h, ctypes.byref(ca), ctypes.byref(co),
                                           _stream()), "secpe_bootstrap_batch")
        out.update(co)
        return out

    def close(self):
        if self.h:
            lib().secpe_boot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def argmax_batch_boot(ctx, keys, boot, queries):
    """secpe_argmax_batch_boot: argmax_batch with every refresh a bootstrap."""
    qarr, keep = _query_array(queries)
    _check(lib().secpe_argmax_batch_boot(ctx.h, keys.h, boot.h, qarr, len(queries), _stream()),
           "secpe_argmax_batch_boot")
    for q, (_, z) in zip(queries, keep):
        q["z_out"].update(z)


class Graph:
    """One CUDA graph of a whole batched Argmax (secpe_argmax_batch_capture).
    It keeps the device addresses of the queries' ciphertexts, z_out buffers
    and keys: the caller keeps those tensors alive while the graph is used."""

    def __init__(self, ctx, keys, queries):
        qarr, keep = _query_array(queries)
        h = ctypes.c_void_p()
        nodes = ctypes.c_int64()
        _check(lib().secpe_argmax_batch_capture(ctx.h, keys.h, qarr, len(queries), ctypes.byref(h),
                                                ctypes.byref(nodes)), "secpe_argmax_batch_capture")
        self.h = h
        self.nodes = int(nodes.value)
        self._refs = (ctx, keys)
        for q, (_, z) in zip(queries, keep):
            q["z_out"].update(z)

    def launch(self):
        _check(lib().secpe_graph_launch(self.h, _stream()), "secpe_graph_launch")

    def close(self):
        if getattr(self, "h", None):
            lib().secpe_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ batched primitives
class CtBatch:
    """`batch` ciphertexts in one tensor [batch][2][cap][N] at a common level/scale."""

    def __init__(self, data, level, scale):
        self.data = data
        self.level = level
        self.scale = scale

    @property
    def batch(self):
        return int(self.data.shape[0])

    def struct(self):
        cap, n = int(self.data.shape[2]), int(self.data.shape[3])
        return CtBatchC(ctypes.c_void_p(self.data.data_ptr()), self.batch, cap, self.level, self.scale, 2 * cap * n)

    def update(self, c):
        self.level = int(c.level)
        self.scale = float(c.scale)


def keyswitch_batch(ctx, keys, galois_step, d, out):
    cd, co = d.struct(), out.struct()
    _check(lib().secpe_keyswitch_batch(ctx.h, keys.h, galois_step, ctypes.byref(cd), ctypes.byref(co), _stream()),
           "secpe_keyswitch_batch")
    out.update(co)
    return out


def keyswitch_batch_tc(ctx, keys, galois_step, d, out):
    """Precision variant of keyswitch_batch (tensor-pipe transforms and key
    inner product); bit-identical to it."""
    cd, co = d.struct(), out.struct()
    _check(lib().secpe_keyswitch_batch_tc(ctx.h, keys.h, galois_step, ctypes.byref(cd), ctypes.byref(co),
                                          _stream()), "secpe_keyswitch_batch_tc")
    out.update(co)
    return out


def mul_relin_batch(ctx, keys, a, b, out):
    ca, cb, co = a.struct(), b.struct(), out.struct()
    _check(lib().secpe_mul_relin_batch(ctx.h, keys.h, ctypes.byref(ca), ctypes.byref(cb), ctypes.byref(co),
                                       _stream()), "secpe_mul_relin_batch")
    out.update(co)
    return out


def rotate_batch(ctx, keys, a, steps, out):
    ca, co = a.struct(), out.struct()
    _check(lib().secpe_rotate_batch(ctx.h, keys.h, ctypes.byref(ca), steps, ctypes.byref(co), _stream()),
           "secpe_rotate_batch")
    out.update(co)
    return out


def rescale_batch(ctx, a, out):
    ca, co = a.struct(), out.struct()
    _check(lib().secpe_rescale_batch(ctx.h, ctypes.byref(ca), ctypes.byref(co), _stream()), "secpe_rescale_batch")
    out.update(co)
    return out


# ------------------------------------------------------------------ server
class Server:
    """Continuous-batching server (secpe_server_*).  Keeps the ctypes query
    structs of submitted queries alive until they are forgotten."""

    def __init__(self, ctx, keys, hbm_budget_bytes, max_batch=64):
        h = ctypes.c_void_p()
        _check(lib().secpe_server_create(ctx.h, keys.h, int(hbm_budget_bytes), max_batch, ctypes.byref(h)),
               "secpe_server_create")
        self.h, self.ctx, self.keys = h, ctx, keys
        self._keep = {}

    def submit(self, cts, C, d_min, d_max, qseed, z_out, keys=None):
        """keys: the query's tenant key set (default: the server's)."""
        arr = (CtC * len(cts))(*[c.struct() for c in cts])
        z = z_out.struct()
        qc = QueryC(arr, len(cts), C, d_min, d_max, qseed, ctypes.pointer(z),
                    keys.h.value if keys is not None else None)
        t = ctypes.c_int64()
        _check(lib().secpe_server_submit(self.h, ctypes.byref(qc), ctypes.byref(t)), "secpe_server_submit")
        self._keep[t.value] = (arr, z, qc, z_out, cts, keys)
        return t.value

    def step(self):
        n = ctypes.c_int32()
        _check(lib().secpe_server_step(self.h, _stream(), ctypes.byref(n)), "secpe_server_step")
        return n.value

    def poll(self, ticket):
        d = ctypes.c_int32()
        _check(lib().secpe_server_poll(self.h, ticket, ctypes.byref(d)), "secpe_server_poll")
        if d.value == 1:
            z, z_out = self._keep[ticket][1], self._keep[ticket][3]
            z_out.update(z)
        return d.value

    def wait(self, ticket, timeout_s=600.0):
        _check(lib().secpe_server_wait(self.h, ticket, timeout_s), "secpe_server_wait")
        return self.poll(ticket)

    def cancel(self, ticket):
        _check(lib().secpe_server_cancel(self.h, ticket), "secpe_server_cancel")

    def forget(self, ticket):
        _check(lib().secpe_server_forget(self.h, ticket), "secpe_server_forget")
        self._keep.pop(ticket, None)

    def stats(self):
        st = ServerStatsC()
        _check(lib().secpe_server_stats(self.h, ctypes.byref(st)), "secpe_server_stats")
        return {f[0]: int(getattr(st, f[0])) for f in ServerStatsC._fields_}

    def close(self):
        if self.h:
            lib().secpe_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ntt32:
    """secpe_ntt32: the word-size probe's twiddle table for 32-bit primes
    (q < 2^30, q = 1 mod 2N, N = 2^16); limbs are uint32 torch tensors."""

    def __init__(self, primes, log_n=16):
        arr = (ctypes.c_uint32 * len(primes))(*primes)
        h = ctypes.c_void_p()
        _check(lib().secpe_ntt32_create(log_n, arr, len(primes), ctypes.byref(h)), "secpe_ntt32_create")
        self.h, self.primes = h, list(primes)

    @staticmethod
    def _idx(idx):
        return (ctypes.c_int32 * len(idx))(*idx)

    def ntt(self, limbs, prime_idx, inverse=False):
        """In place on limbs [count][N] (a contiguous uint32 device tensor)."""
        _check(lib().secpe_ntt32(self.h, ctypes.c_void_p(limbs.data_ptr()), self._idx(prime_idx), len(prime_idx),
                                 int(inverse), _stream()), "secpe_ntt32")

    def bconv(self, x, in_idx, out, out_idx):
        """x [batch][n_in][N] -> out [batch][n_out][N] (uint32 device tensors)."""
        _check(lib().secpe_bconv32(self.h, ctypes.c_void_p(x.data_ptr()), self._idx(in_idx), len(in_idx),
                                   ctypes.c_void_p(out.data_ptr()), self._idx(out_idx), len(out_idx), x.shape[0],
                                   _stream()), "secpe_bconv32")

    def keyswitch(self, d, q_idx, p_idx, alpha, key, out, fused=True):
        """d [batch][nq][N] -> out [batch][2][nq][N] with key [dnum][2][nq+np][N] (uint32 device tensors)."""
        _check(lib().secpe_keyswitch32(self.h, ctypes.c_void_p(d.data_ptr()), self._idx(q_idx), len(q_idx),
                                       self._idx(p_idx), len(p_idx), alpha, ctypes.c_void_p(key.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), d.shape[0], int(fused), _stream()),
               "secpe_keyswitch32")

    def close(self):
        if self.h:
            lib().secpe_ntt32_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
