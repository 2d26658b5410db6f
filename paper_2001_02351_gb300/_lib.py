"""ctypes binding of librespack_gb300.so: argument marshalling only.

Every function of the C ABI (include/respack_gb300.h) has a method of the same name on
`Context`.  Arrays are either numpy arrays (host, synchronous call) or CUDA torch
tensors (device, queued on torch's current stream).  Nothing here computes any step
of the method; a missing library raises instead of falling back to anything.
"""
import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "librespack_gb300.so")

RP_OK, RP_ERR_ARG, RP_ERR_STATE, RP_ERR_OOM, RP_ERR_CUDA, RP_ERR_NUMERIC, RP_ERR_TIMEOUT, RP_ERR_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
RP_FP64_NATIVE, RP_FP64_EMULATED, RP_TF32X3, RP_BF16X3 = 0, 1, 2, 3
RP_AXIS_REAL, RP_AXIS_IMAG = 0, 1
TILE_WIDTHS = (160, 192, 208, 224, 256)     # raw rows per tile of the BF16x3 contraction kernel
RP_TIME_ORDERED, RP_RETARDED = 0, 1

_STATUS = {0: "RP_OK", -1: "RP_ERR_ARG", -2: "RP_ERR_STATE", -3: "RP_ERR_OOM", -4: "RP_ERR_CUDA",
           -5: "RP_ERR_NUMERIC", -6: "RP_ERR_TIMEOUT", -7: "RP_ERR_UNSUPPORTED"}

# every symbol the header declares
EXPORTS = ["rp_setup_cell", "rp_load_bands", "rp_sphere_size", "rp_pair_density", "rp_tetra_weights",
           "rp_contract_chi0", "rp_build_chi0", "rp_solve_w", "rp_check_numeric", "rp_profile_enable",
           "rp_profile_read", "rp_last_error", "rp_destroy", "rp_contract_chi0_static", "rp_sphere_size_at",
           "rp_build_chi0_batched", "rp_solve_w_batched", "rp_set_wait_limit", "rp_set_pair_budget", "rp_contract_chi0_static_status",
           "rp_build_chi0_kset", "rp_tune_contraction", "rp_set_contraction_tile",
           "rp_load_wannier", "rp_interaction", "rp_build_chi0_q0", "rp_solve_w_q0", "rp_optics",
           "rp_rotate_q", "rp_probe_peaks", "rp_plasma", "rp_transform_grid", "rp_set_fermi",
           "rp_set_dyson_hermitian"]


class RPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: run paper_2001_02351_gb300.build.build() first")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "rp_setup_cell": (I, [P, P, P, D, D, ctypes.POINTER(P)]),
        "rp_load_bands": (I, [P, I, I, I, P, I, P, P, P, P]),
        "rp_sphere_size": (I, [P, P, ctypes.POINTER(I), ctypes.POINTER(I), P, P]),
        "rp_transform_grid": (I, [P, P, P, ctypes.POINTER(I)]),
        "rp_pair_density": (I, [P, P, I, I, P, I, P]),
        "rp_tetra_weights": (I, [P, P, I, I, I, P, D, D, D, I, P, I, P]),
        "rp_contract_chi0": (I, [P, I, LL, I, P, P, I, P, I, P]),
        "rp_build_chi0": (I, [P, P, I, I, I, P, D, D, D, I, P, I, P]),
        "rp_solve_w": (I, [P, P, I, P, P, P, I, P]),
        "rp_check_numeric": (I, [P]),
        "rp_profile_enable": (I, [P, I]),
        "rp_profile_read": (I, [P, P, P]),
        "rp_last_error": (ctypes.c_char_p, [P]),
        "rp_destroy": (None, [P]),
        "rp_contract_chi0_static": (I, [I, LL, I, P, P, P, P]),
        "rp_sphere_size_at": (I, [P, P, D, ctypes.POINTER(I), ctypes.POINTER(I), P, P]),
        "rp_build_chi0_batched": (I, [P, I, P, P, I, I, I, P, D, D, D, I, P, I, P]),
        "rp_solve_w_batched": (I, [P, I, P, P, I, P, P, P, I, P]),
        "rp_set_wait_limit": (I, [P, LL]),
        "rp_set_pair_budget": (I, [P, LL]),
        "rp_set_fermi": (I, [P, ctypes.c_double]),
        "rp_set_dyson_hermitian": (I, [P, I]),
        "rp_build_chi0_kset": (I, [P, P, I, P, I, I, I, P, D, D, D, I, P, I, P]),
        "rp_tune_contraction": (I, [P, I, LL, I, ctypes.POINTER(I), P]),
        "rp_set_contraction_tile": (I, [P, I, I]),
        "rp_load_wannier": (I, [P, I, P]),
        "rp_build_chi0_q0": (I, [P, P, I, I, I, P, D, D, D, I, P, I, P]),
        "rp_solve_w_q0": (I, [P, I, P, P, P, I, P]),
        "rp_optics": (I, [P, I, P, P, P]),
        "rp_rotate_q": (I, [P, P, P, P, I, P, P, I, P]),
        "rp_probe_peaks": (I, [P]),
        "rp_plasma": (I, [P, D, P]),
        "rp_interaction": (I, [P, P, I, P, I, P, P, P, I, I, P]),
        "rp_contract_chi0_static_status": (I, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _dev_ptr(t):
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("device arrays must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """One crystal + k mesh + band set (rp_ctx)."""

    def __init__(self, lat, kmesh, fft, ecut_psi, ecut_eps):
        self._lib = library()
        self._h = ctypes.c_void_p()
        lat_, plat = _host(np.asarray(lat, dtype=np.float64).reshape(9), np.float64)
        km_, pkm = _host(kmesh, np.int32)
        ff_, pff = _host(fft, np.int32)
        code = self._lib.rp_setup_cell(plat, pkm, pff, float(ecut_psi), float(ecut_eps), ctypes.byref(self._h))
        if code != RP_OK:
            raise RPError(code, "rp_setup_cell rejected its arguments")
        self._keep = (lat_, km_, ff_)

    # -- helpers -------------------------------------------------------------------------
    def _check(self, code):
        if code != RP_OK:
            raise RPError(code, self._lib.rp_last_error(self._h).decode())

    def close(self):
        if self._h:
            self._lib.rp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI ---------------------------------------------------------------------------
    def rp_load_bands(self, nocc, npw, miller, coef, energy, T=None):
        coef = np.ascontiguousarray(coef, dtype=np.complex128)
        nk, nband, npw_max = coef.shape
        npw_, pnpw = _host(npw, np.int32)
        mil_, pmil = _host(np.asarray(miller).reshape(nk, npw_max, 3), np.int32)
        en_, pen = _host(energy, np.float64)
        pT = None
        if T is not None:
            T_, pT = _host(T, np.float64)
        self._check(self._lib.rp_load_bands(self._h, nk, nband, int(nocc), pnpw, npw_max, pmil,
                                            coef.ctypes.data_as(ctypes.c_void_p), pen, pT))
        self.nk, self.nband, self.nocc, self.nemp = nk, nband, int(nocc), nband - int(nocc)

    load_bands = rp_load_bands

    def rp_sphere_size(self, q, ecut_eps=None):
        """(Miller [NG][3], tail [N_tail][3]) of q, with the context's cut-off or ecut_eps (Ha)."""
        q_, pq = _host(q, np.float64)
        ng, nt = ctypes.c_int(), ctypes.c_int()
        if ecut_eps is None:
            call = lambda g_, t_: self._lib.rp_sphere_size(self._h, pq, ctypes.byref(ng), ctypes.byref(nt), g_, t_)
        else:
            call = lambda g_, t_: self._lib.rp_sphere_size_at(self._h, pq, float(ecut_eps), ctypes.byref(ng),
                                                              ctypes.byref(nt), g_, t_)
        self._check(call(None, None))
        g = np.zeros((ng.value, 3), dtype=np.int32)
        t = np.zeros((max(nt.value, 1), 3), dtype=np.int32)
        self._check(call(g.ctypes.data_as(ctypes.c_void_p), t.ctypes.data_as(ctypes.c_void_p)))
        return g, t[:nt.value]

    rp_sphere_size_at = rp_sphere_size

    def rp_transform_grid(self, q):
        """((N1, N2, N3), window half-width) of the pair transforms of q."""
        q_, pq = _host(q, np.float64)
        n = np.zeros(3, dtype=np.int32)
        w = ctypes.c_int()
        self._check(self._lib.rp_transform_grid(self._h, pq, n.ctypes.data_as(ctypes.c_void_p), ctypes.byref(w)))
        return tuple(int(x) for x in n), w.value

    def _out(self, out, shape, dtype=np.complex128):
        if out is None:
            return np.zeros(shape, dtype=dtype), 0
        return out, (1 if _is_torch(out) else 0)

    def _ptr(self, a, on_device):
        return _dev_ptr(a) if on_device else a.ctypes.data_as(ctypes.c_void_p)

    def rp_pair_density(self, q, k_begin, k_end, out=None):
        g, _ = self.rp_sphere_size(q)
        K = (k_end - k_begin) * self.nemp * self.nocc
        out, dev = self._out(out, (len(g), K))
        q_, pq = _host(q, np.float64)
        self._check(self._lib.rp_pair_density(self._h, pq, int(k_begin), int(k_end), self._ptr(out, dev), dev,
                                              _stream() if dev else None))
        return out

    def rp_tetra_weights(self, q, axis, ordering, freq, delta, delta_a=1e-8, delta_r=1e-8, out=None,
                         precision=RP_FP64_NATIVE):
        fr, pf = _host(freq, np.float64)
        K = self.nk * self.nemp * self.nocc
        out, dev = self._out(out, (len(fr), K))
        q_, pq = _host(q, np.float64)
        self._check(self._lib.rp_tetra_weights(self._h, pq, int(axis), int(ordering), len(fr), pf, float(delta),
                                               float(delta_a), float(delta_r), int(precision), self._ptr(out, dev), dev,
                                               _stream() if dev else None))
        return out

    def rp_contract_chi0(self, M, w, precision=RP_FP64_NATIVE, out=None):
        dev = 1 if _is_torch(M) else 0
        if dev:
            ng, K = M.shape
            nf = w.shape[0]
            if out is None:
                import torch
                out = torch.empty((nf, ng, ng), dtype=torch.complex128, device=M.device)
            pm, pw = _dev_ptr(M), _dev_ptr(w)
        else:
            M = np.ascontiguousarray(M, dtype=np.complex128)
            w = np.ascontiguousarray(w, dtype=np.complex128)
            ng, K = M.shape
            nf = w.shape[0]
            out = np.zeros((nf, ng, ng), dtype=np.complex128) if out is None else out
            pm, pw = M.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p)
        self._check(self._lib.rp_contract_chi0(self._h, int(ng), int(K), int(nf), pm, pw, int(precision),
                                               self._ptr(out, dev), dev, _stream() if dev else None))
        return out

    def rp_build_chi0(self, q, axis, ordering, freq, delta, precision=RP_FP64_NATIVE, delta_a=1e-8,
                      delta_r=1e-8, out=None):
        g, _ = self.rp_sphere_size(q)
        fr, pf = _host(freq, np.float64)
        out, dev = self._out(out, (len(fr), len(g), len(g)))
        q_, pq = _host(q, np.float64)
        self._check(self._lib.rp_build_chi0(self._h, pq, int(axis), int(ordering), len(fr), pf, float(delta),
                                            float(delta_a), float(delta_r), int(precision), self._ptr(out, dev),
                                            dev, _stream() if dev else None))
        return out

    def rp_build_chi0_kset(self, q, k_list, axis, ordering, freq, delta, precision=RP_FP64_NATIVE, delta_a=1e-8,
                           delta_r=1e-8, out=None):
        """chi0 of q summed over the pairs of the mesh points k_list only (full-mesh weights)."""
        g, _ = self.rp_sphere_size(q)
        fr, pf = _host(freq, np.float64)
        ks, pk = _host(k_list, np.int32)
        out, dev = self._out(out, (len(fr), len(g), len(g)))
        q_, pq = _host(q, np.float64)
        self._check(self._lib.rp_build_chi0_kset(self._h, pq, len(ks), pk, int(axis), int(ordering), len(fr), pf,
                                                 float(delta), float(delta_a), float(delta_r), int(precision),
                                                 self._ptr(out, dev), dev, _stream() if dev else None))
        return out

    def rp_build_chi0_batched(self, qs, axis, ordering, freq, delta, precision=RP_FP64_NATIVE, ecut_eps=None,
                              delta_a=1e-8, delta_r=1e-8, outs=None):
        """chi0 of every q of qs [nq][3] (per-q cut-offs ecut_eps [nq] or None); a list of arrays
        (host) or of the given CUDA tensors."""
        qs_, pq = _host(np.asarray(qs, dtype=np.float64).reshape(-1, 3), np.float64)
        nq = qs_.shape[0]
        cuts = None if ecut_eps is None else np.ascontiguousarray(ecut_eps, dtype=np.float64)
        fr, pf = _host(freq, np.float64)
        if outs is None:
            outs = []
            for i in range(nq):
                g, _ = self.rp_sphere_size(qs_[i], None if cuts is None else cuts[i])
                outs.append(np.zeros((len(fr), len(g), len(g)), dtype=np.complex128))
        dev = 1 if _is_torch(outs[0]) else 0
        ptrs = (ctypes.c_void_p * nq)(*[self._ptr(o, dev).value for o in outs])
        self._check(self._lib.rp_build_chi0_batched(
            self._h, nq, pq, None if cuts is None else cuts.ctypes.data_as(ctypes.c_void_p), int(axis), int(ordering),
            len(fr), pf, float(delta), float(delta_a), float(delta_r), int(precision), ptrs, dev,
            _stream() if dev else None))
        return outs

    def rp_solve_w_batched(self, qs, chi0s, ecut_eps=None, outs=None):
        """W of every member of a batch: list of (W, tail) for host arrays; for CUDA tensors W is
        written into the tensors of `outs` (no tails) and those are returned."""
        qs_, pq = _host(np.asarray(qs, dtype=np.float64).reshape(-1, 3), np.float64)
        nq = qs_.shape[0]
        cuts = None if ecut_eps is None else np.ascontiguousarray(ecut_eps, dtype=np.float64)
        if _is_torch(chi0s[0]):
            import torch
            outs = [torch.empty_like(c) for c in chi0s] if outs is None else outs
            P = ctypes.c_void_p
            pc = (P * nq)(*[_dev_ptr(c).value for c in chi0s])
            pw = (P * nq)(*[_dev_ptr(w).value for w in outs])
            self._check(self._lib.rp_solve_w_batched(self._h, nq, pq,
                                                     None if cuts is None else cuts.ctypes.data_as(P),
                                                     int(chi0s[0].shape[0]), pc, pw, None, 1, _stream()))
            return outs
        chis = [np.ascontiguousarray(c, dtype=np.complex128) for c in chi0s]
        Ws = [np.zeros_like(c) for c in chis]
        tails = []
        for i in range(nq):
            _, t = self.rp_sphere_size(qs_[i], None if cuts is None else cuts[i])
            tails.append(np.zeros(max(len(t), 1)))
        P = ctypes.c_void_p
        pc = (P * nq)(*[c.ctypes.data for c in chis])
        pw = (P * nq)(*[w.ctypes.data for w in Ws])
        pt = (P * nq)(*[t.ctypes.data for t in tails])
        self._check(self._lib.rp_solve_w_batched(self._h, nq, pq, None if cuts is None else cuts.ctypes.data_as(P),
                                                 int(chis[0].shape[0]), pc, pw, pt, 0, None))
        out = []
        for i in range(nq):
            _, t = self.rp_sphere_size(qs_[i], None if cuts is None else cuts[i])
            out.append((Ws[i], tails[i][:len(t)]))
        return out

    def rp_solve_w(self, q, chi0, out=None, tail=None):
        g, t = self.rp_sphere_size(q)
        dev = 1 if _is_torch(chi0) else 0
        nf = chi0.shape[0]
        if dev:
            import torch
            out = torch.empty_like(chi0) if out is None else out
            tail = torch.zeros(max(len(t), 1), dtype=torch.float64, device=chi0.device) if tail is None else tail
            pc = _dev_ptr(chi0)
        else:
            chi0 = np.ascontiguousarray(chi0, dtype=np.complex128)
            out = np.zeros_like(chi0) if out is None else out
            tail = np.zeros(max(len(t), 1)) if tail is None else tail
            pc = chi0.ctypes.data_as(ctypes.c_void_p)
        q_, pq = _host(q, np.float64)
        self._check(self._lib.rp_solve_w(self._h, pq, int(nf), pc, self._ptr(out, dev), self._ptr(tail, dev), dev,
                                         _stream() if dev else None))
        return out, tail[:len(t)]

    def rp_check_numeric(self):
        self._check(self._lib.rp_check_numeric(self._h))

    def rp_build_chi0_q0(self, qhat, axis, ordering, freq, delta, precision=RP_FP64_NATIVE, delta_a=1e-8,
                         delta_r=1e-8, out=None):
        """Extended chi0 [nfreq][NG+1][NG+1] at q -> 0 along qhat (index 0: head and wings)."""
        g, _ = self.rp_sphere_size(np.zeros(3))
        fr, pf = _host(freq, np.float64)
        out, dev = self._out(out, (len(fr), len(g) + 1, len(g) + 1))
        qh, pq = _host(qhat, np.float64)
        self._check(self._lib.rp_build_chi0_q0(self._h, pq, int(axis), int(ordering), len(fr), pf, float(delta),
                                               float(delta_a), float(delta_r), int(precision), self._ptr(out, dev),
                                               dev, _stream() if dev else None))
        return out

    def rp_solve_w_q0(self, chi0, out=None):
        """W of the extended q -> 0 matrix (W[f][0][0] = (4 pi/Omega) eps^-1_00)."""
        dev = 1 if _is_torch(chi0) else 0
        if dev:
            import torch
            out = torch.empty_like(chi0) if out is None else out
            pc = _dev_ptr(chi0)
        else:
            chi0 = np.ascontiguousarray(chi0, dtype=np.complex128)
            out = np.zeros_like(chi0) if out is None else out
            pc = chi0.ctypes.data_as(ctypes.c_void_p)
        self._check(self._lib.rp_solve_w_q0(self._h, int(chi0.shape[0]), pc, self._ptr(out, dev), None, dev,
                                            _stream() if dev else None))
        return out

    def rp_rotate_q(self, q_irr, q, S, X_irr, out=None):
        """X at q from X_irr at q_irr under the integer rotation S (k -> k S)."""
        qi, pqi = _host(q_irr, np.float64)
        q_, pq = _host(q, np.float64)
        S_, pS = _host(np.asarray(S).reshape(9), np.int32)
        dev = 1 if _is_torch(X_irr) else 0
        if dev:
            import torch
            out = torch.empty_like(X_irr) if out is None else out
            px = _dev_ptr(X_irr)
        else:
            X_irr = np.ascontiguousarray(X_irr, dtype=np.complex128)
            out = np.zeros_like(X_irr) if out is None else out
            px = X_irr.ctypes.data_as(ctypes.c_void_p)
        self._check(self._lib.rp_rotate_q(self._h, pqi, pq, pS, int(X_irr.shape[0]), px, self._ptr(out, dev), dev,
                                          _stream() if dev else None))
        return out

    def rp_plasma(self, fermi):
        """(w_pl^2)^{mu nu} [3, 3] of Eq. plasma at the Fermi energy `fermi` (Ha)."""
        out = np.zeros(9)
        self._check(self._lib.rp_plasma(self._h, float(fermi), out.ctypes.data_as(ctypes.c_void_p)))
        return out.reshape(3, 3)

    def rp_optics(self, freq, W00):
        """[nfreq][5]: Re eps_M, Im eps_M, loss function, Re sigma, reflectivity."""
        fr, pf = _host(freq, np.float64)
        w_, pw = _host(W00, np.complex128)
        out = np.zeros((len(fr), 5))
        self._check(self._lib.rp_optics(self._h, len(fr), pf, pw, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def rp_load_wannier(self, coef):
        """coef [nk][nw][npw_max]: plane-wave coefficients of the Wannier functions' Bloch orbitals."""
        coef = np.ascontiguousarray(coef, dtype=np.complex128)
        self._check(self._lib.rp_load_wannier(self._h, int(coef.shape[1]), coef.ctypes.data_as(ctypes.c_void_p)))
        self.nw = int(coef.shape[1])

    def rp_interaction(self, q, R_list, W=None, U=None, J=None, accumulate=False):
        """This q's term of U_{i0jR}, J_{i0jR} [nfreq][nR][nw][nw] (bare when W is None); host arrays, or
        CUDA tensors when W (or U) is one.  With accumulate the term is added to the given U, J."""
        R_, pR = _host(np.asarray(R_list).reshape(-1, 3), np.int32)
        nR = R_.shape[0]
        dev = 1 if (_is_torch(W) or _is_torch(U)) else 0
        nf = 1 if W is None else W.shape[0]
        shape = (nf, nR, self.nw, self.nw)
        if dev:
            import torch
            U = torch.zeros(shape, dtype=torch.complex128, device="cuda") if U is None else U
            J = torch.zeros(shape, dtype=torch.complex128, device="cuda") if J is None else J
            pW = None if W is None else _dev_ptr(W)
        else:
            U = np.zeros(shape, dtype=np.complex128) if U is None else U
            J = np.zeros(shape, dtype=np.complex128) if J is None else J
            if W is not None:
                W = np.ascontiguousarray(W, dtype=np.complex128)
            pW = None if W is None else W.ctypes.data_as(ctypes.c_void_p)
        q_, pq = _host(q, np.float64)
        self._check(self._lib.rp_interaction(self._h, pq, int(nf), pW, nR, pR, self._ptr(U, dev), self._ptr(J, dev),
                                             1 if accumulate else 0, dev, _stream() if dev else None))
        return U, J

    def rp_tune_contraction(self, ng, K, nfreq):
        """(chosen BN, {BN: ms}) for BF16x3 contractions of this shape; the choice is kept in the context."""
        bn = ctypes.c_int()
        ms = np.zeros(5)
        self._check(self._lib.rp_tune_contraction(self._h, int(ng), int(K), int(nfreq), ctypes.byref(bn),
                                                  ms.ctypes.data_as(ctypes.c_void_p)))
        return bn.value, dict(zip(TILE_WIDTHS, ms.tolist()))

    def rp_set_contraction_tile(self, ng, bn):
        self._check(self._lib.rp_set_contraction_tile(self._h, int(ng), int(bn)))

    def tuned_tile(self, ng, K, nfreq, cache_path=None):
        """The contraction tile for this shape from a JSON cache keyed by device and shape, tuned and
        written back when missing (argument handling only; the timing runs in the library)."""
        import json
        import torch
        key = f"{torch.cuda.get_device_name()}|ng={int(ng)}|K={int(K)}|nf={int(nfreq)}"
        cache = {}
        if cache_path and os.path.exists(cache_path):
            try:
                cache = json.load(open(cache_path))
            except (OSError, ValueError):
                cache = {}
        if key in cache:
            self.rp_set_contraction_tile(ng, cache[key]["bn"])
            return cache[key]["bn"], cache[key]["ms"]
        bn, ms = self.rp_tune_contraction(ng, K, nfreq)
        if cache_path:
            cache[key] = {"bn": bn, "ms": {str(k): v for k, v in ms.items()}}
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            tmp = cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(tmp, cache_path)
        return bn, ms

    def rp_set_wait_limit(self, limit_ns):
        self._check(self._lib.rp_set_wait_limit(self._h, int(limit_ns)))

    def rp_set_fermi(self, efermi=float("nan")):
        """Fermi energy (Ha) of a metal: Fermi-surface clipping of the weights; NaN turns it off."""
        self._check(self._lib.rp_set_fermi(self._h, float(efermi)))

    def rp_set_dyson_hermitian(self, on=True):
        """Dyson steps by the Hermitian positive definite sweep (imaginary axis) or pivoted Gauss-Jordan."""
        self._check(self._lib.rp_set_dyson_hermitian(self._h, 1 if on else 0))

    def rp_set_pair_budget(self, nbytes):
        self._check(self._lib.rp_set_pair_budget(self._h, int(nbytes)))

    def rp_profile_enable(self, enable=True):
        self._check(self._lib.rp_profile_enable(self._h, 1 if enable else 0))

    def rp_profile_read(self):
        """(ms[6], launches[6]) per stage: gather+inverse, pair forward, weights, contraction kernel,
        Dyson, split-contraction operands (bf16 split of M, float weights)."""
        ms = np.zeros(6)
        nl = np.zeros(6, dtype=np.int64)
        self._check(self._lib.rp_profile_read(self._h, ms.ctypes.data_as(ctypes.c_void_p),
                                              nl.ctypes.data_as(ctypes.c_void_p)))
        return ms, nl


def probe_peaks():
    """Measured TFLOP/s of the current device: FP64 FMA, FP64 mma.sync, bf16 tcgen05 (rp_probe_peaks)."""
    lib = library()
    out = np.zeros(3)
    code = lib.rp_probe_peaks(out.ctypes.data_as(ctypes.c_void_p))
    if code != RP_OK:
        raise RPError(code, "rp_probe_peaks failed")
    return {"fp64_fma": float(out[0]), "fp64_mma": float(out[1]), "bf16_tcgen05": float(out[2])}


def context_for(wl, q_index=0):
    """Context with the bands of a synthetic workload loaded (helper for tests and bench)."""
    b = wl.bands
    ctx = Context(b.cell.lat, b.kmesh, wl.fft, b.ecut_psi, float(wl.ecut_eps[q_index]))
    nb = wl.nocc + wl.nemp
    ctx.load_bands(wl.nocc, b.npw, b.miller, b.coef[:, :nb], b.energy[:, :nb],
                   None if wl.T is None else wl.T[:, :nb])
    return ctx
