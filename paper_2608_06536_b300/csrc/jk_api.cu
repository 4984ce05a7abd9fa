// C ABI of libjk.so: handle, arena, validation and dispatch (see include/jk.h).
#include <cstdarg>
#include <cstring>
#include <new>

#include "jk_internal.h"

namespace jk {

jk_status set_error(jk_ctx *h, jk_status s, const char *fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->last_error = buf;
    }
    return s;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// True if p is memory the current device can read (device or managed).
static bool device_readable(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Validate one molecule and fill a Problem; h may be NULL (query path).
static jk_status make_problem(jk_ctx *h, const jk_factor *f, int nd,
                              const jk_density *d, bool check_ptrs, Problem &pb) {
    if (!f || !d) return set_error(h, JK_ERR_ARG, "factor or density array is NULL");
    if (f->nbf < 1 || f->naux < 1)
        return set_error(h, JK_ERR_SHAPE, "nbf=%d naux=%d must be >= 1", f->nbf, f->naux);
    if (f->nbf > 65535)
        return set_error(h, JK_ERR_SHAPE, "nbf=%d exceeds 65535", f->nbf);
    if (nd < 1 || nd > kMaxDens)
        return set_error(h, JK_ERR_SHAPE, "nd=%d must be in [1, %d]", nd, kMaxDens);
    pb.n = f->nbf;
    pb.naux = f->naux;
    pb.nd = nd;
    pb.L = f->L;
    int c = 0, ks = 0, km = 0;
    for (int s = 0; s < nd; s++) {
        if (d[s].k < 1 || d[s].k > f->nbf * 4)
            return set_error(h, JK_ERR_SHAPE, "density %d: k=%d out of range [1, 4*nbf]", s, d[s].k);
        pb.k[s] = d[s].k;
        pb.sym[s] = d[s].symmetric ? 1 : 0;
        pb.X[s] = d[s].X;
        pb.Y[s] = d[s].symmetric ? d[s].X : d[s].Y;
        pb.offX[s] = c;
        c += d[s].k;
        if (pb.sym[s]) {
            pb.offY[s] = pb.offX[s];
        } else {
            pb.offY[s] = c;
            c += d[s].k;
        }
        ks += d[s].k;
        if (d[s].k > km) km = d[s].k;
    }
    pb.ctot = c;
    pb.ksum = ks;
    pb.kmax = km;
    if (check_ptrs) {
        if (!f->L) return set_error(h, JK_ERR_ARG, "factor L is NULL");
        if (!aligned16(f->L)) return set_error(h, JK_ERR_ARG, "factor L is not 16-byte aligned");
        if (!device_readable(f->L)) return set_error(h, JK_ERR_ARG, "factor L is not device memory");
        for (int s = 0; s < nd; s++) {
            if (!d[s].X || (!d[s].symmetric && !d[s].Y))
                return set_error(h, JK_ERR_ARG, "density %d: X or Y is NULL", s);
            if (!aligned16(d[s].X) || (!d[s].symmetric && !aligned16(d[s].Y)))
                return set_error(h, JK_ERR_ARG, "density %d: X or Y is not 16-byte aligned", s);
            if (!device_readable(d[s].X) || (!d[s].symmetric && !device_readable(d[s].Y)))
                return set_error(h, JK_ERR_ARG, "density %d: X or Y is not device memory", s);
        }
    }
    return JK_OK;
}

static size_t flags_bytes() { return align_up(sizeof(DeviceFlags)); }

static void apply_options(jk_ctx *h, Problem &pb) {
    if (h) pb.aux_chunk = h->aux_chunk;
}

static jk_status check_out(jk_ctx *h, const void *p, const char *what) {
    if (!p) return JK_OK;
    if (!aligned16(p)) return set_error(h, JK_ERR_ARG, "%s is not 16-byte aligned", what);
    if (!device_readable(p)) return set_error(h, JK_ERR_ARG, "%s is not device memory", what);
    return JK_OK;
}

static jk_status begin_call(jk_ctx *h) {
    if (!h) return JK_ERR_ARG;
    h->last_error.clear();
    h->arena.reset(flags_bytes());
    int dev = -1;
    JK_CUDA_TRY(h, cudaGetDevice(&dev));
    if (dev != h->device)
        return set_error(h, JK_ERR_ARG, "handle was created on device %d, current device is %d",
                         h->device, dev);
    return JK_OK;
}

static size_t build_bytes(const Problem &pb, jk_precision p) {
    return p == JK_FP64 ? fp64_build_workspace(pb, fp64_default_pchunk(pb))
                        : split_build_workspace(pb);
}

static size_t adjoint_bytes(const Problem &pb, jk_precision p, bool want_dl) {
    return p == JK_FP64 ? fp64_adjoint_workspace(pb, fp64_default_pchunk(pb), want_dl)
                        : split_adjoint_workspace(pb, want_dl);
}

}  // namespace jk

using namespace jk;

extern "C" {

jk_status jk_create(jk_handle *out, void *workspace, size_t bytes) {
    if (!out) return JK_ERR_ARG;
    *out = nullptr;
    if (!workspace) return JK_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) & (kArenaAlign - 1)) != 0) return JK_ERR_ARG;
    if (bytes < flags_bytes()) return JK_ERR_OOM;
    if (!device_readable(workspace)) return JK_ERR_ARG;
    jk_ctx *h = new (std::nothrow) jk_ctx();
    if (!h) return JK_ERR_OOM;
    h->arena.base = static_cast<char *>(workspace);
    h->arena.bytes = bytes;
    h->flags = reinterpret_cast<DeviceFlags *>(workspace);
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        cudaMemset(h->flags, 0, sizeof(DeviceFlags)) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return JK_ERR_CUDA;
    }
    *out = h;
    return JK_OK;
}

jk_status jk_destroy(jk_handle h) {
    delete h;
    return JK_OK;
}

jk_status jk_workspace_query(jk_op op, int32_t nmol, const jk_factor *f,
                             const int32_t *nd_per_mol, int32_t nd,
                             const jk_density *d, jk_precision p, size_t *bytes) {
    if (!bytes || !f || !d) return JK_ERR_ARG;
    if (p != JK_FP64 && p != JK_SPLIT_BF16) return JK_ERR_ARG;
    size_t need = 0;
    if (op == JK_OP_BATCHED) {
        if (nmol < 1 || !nd_per_mol) return JK_ERR_SHAPE;
        int off = 0;
        std::vector<Problem> pbs(nmol);
        for (int m = 0; m < nmol; m++) {
            jk_status s = make_problem(nullptr, &f[m], nd_per_mol[m], d + off, false, pbs[m]);
            if (s != JK_OK) return s;
            size_t b = build_bytes(pbs[m], p);
            if (b > need) need = b;
            off += nd_per_mol[m];
        }
        if (off != nd) return JK_ERR_SHAPE;
        if (p == JK_SPLIT_BF16) need = split_batched_workspace(nmol, pbs.data());
    } else if (op == JK_OP_BUILD || op == JK_OP_ADJOINT) {
        Problem pb;
        jk_status s = make_problem(nullptr, f, nd, d, false, pb);
        if (s != JK_OK) return s;
        need = op == JK_OP_BUILD ? build_bytes(pb, p) : adjoint_bytes(pb, p, true);
    } else {
        return JK_ERR_ARG;
    }
    *bytes = need + flags_bytes() + kArenaAlign;
    return JK_OK;
}

jk_status jk_build(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d,
                   double *J, double *K, jk_precision p, void *stream) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    Problem pb;
    JK_TRY(make_problem(h, f, nd, d, true, pb));
    apply_options(h, pb);
    JK_TRY(check_out(h, J, "J"));
    JK_TRY(check_out(h, K, "K"));
    if (!J && !K) return JK_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (h->arena.bytes < flags_bytes() + build_bytes(pb, p))
        return set_error(h, JK_ERR_OOM, "arena has %zu bytes, this build needs %zu",
                         h->arena.bytes, flags_bytes() + build_bytes(pb, p));
    const long long n2 = (long long)pb.n * pb.n;
    pb.wantJ = J != nullptr;
    pb.wantK = K != nullptr;
    for (int s = 0; s < nd; s++) {
        pb.J[s] = J ? J + s * n2 : nullptr;
        pb.K[s] = K ? K + s * n2 : nullptr;
    }
    return p == JK_FP64 ? fp64_build(h, pb, st) : split_build(h, pb, st);
}

jk_status jk_build_batched(jk_handle h, int32_t nmol, const jk_factor *f,
                           const int32_t *nd_per_mol, const jk_density *d,
                           double *const *J, double *const *K, jk_precision p,
                           void *stream) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    if (nmol < 1 || !f || !nd_per_mol || !d)
        return set_error(h, JK_ERR_SHAPE, "nmol=%d or a NULL array", nmol);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Validate everything before launching anything.
    std::vector<Problem> pbs(nmol);
    int off = 0;
    for (int m = 0; m < nmol; m++) {
        Problem &pb = pbs[m];
        JK_TRY(make_problem(h, &f[m], nd_per_mol[m], d + off, true, pb));
        apply_options(h, pb);
        pb.wantJ = J != nullptr;
        pb.wantK = K != nullptr;
        for (int s = 0; s < nd_per_mol[m]; s++) {
            pb.J[s] = J ? J[off + s] : nullptr;
            pb.K[s] = K ? K[off + s] : nullptr;
            if (J && !pb.J[s]) return set_error(h, JK_ERR_ARG, "J[%d] is NULL", off + s);
            if (K && !pb.K[s]) return set_error(h, JK_ERR_ARG, "K[%d] is NULL", off + s);
            JK_TRY(check_out(h, pb.J[s], "J[i]"));
            JK_TRY(check_out(h, pb.K[s], "K[i]"));
        }
        if (p == JK_FP64 && h->arena.bytes < flags_bytes() + build_bytes(pb, p))
            return set_error(h, JK_ERR_OOM, "arena too small for molecule %d", m);
        off += nd_per_mol[m];
    }
    if (!J && !K) return JK_OK;
    return batched_build(h, nmol, pbs.data(), p, st);
}

jk_status jk_adjoint(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d,
                     const double *W, const double *V, double *dX, double *dY,
                     double *dL, jk_precision p, void *stream) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    Problem pb;
    JK_TRY(make_problem(h, f, nd, d, true, pb));
    apply_options(h, pb);
    if (!dX || !dY) return set_error(h, JK_ERR_ARG, "dX and dY are required");
    JK_TRY(check_out(h, dX, "dX"));
    JK_TRY(check_out(h, dY, "dY"));
    JK_TRY(check_out(h, dL, "dL"));
    JK_TRY(check_out(h, W, "W"));
    JK_TRY(check_out(h, V, "V"));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    size_t need = flags_bytes() + adjoint_bytes(pb, p, dL != nullptr);
    if (h->arena.bytes < need)
        return set_error(h, JK_ERR_OOM, "arena has %zu bytes, this adjoint needs %zu",
                         h->arena.bytes, need);
    return p == JK_FP64 ? fp64_adjoint(h, pb, W, V, dX, dY, dL, st)
                        : split_adjoint(h, pb, W, V, dX, dY, dL, st);
}

jk_status jk_set_option(jk_handle h, jk_option opt, int64_t value) {
    if (!h) return JK_ERR_ARG;
    if (opt == JK_OPT_AUX_CHUNK) {
        if (value < 0 || value > (1 << 30)) return set_error(h, JK_ERR_ARG, "aux chunk out of range");
        h->aux_chunk = static_cast<int>(value);
        return JK_OK;
    }
    return set_error(h, JK_ERR_ARG, "unknown option %d", (int)opt);
}

jk_status jk_sync_status(jk_handle h, void *stream) {
    if (!h) return JK_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    JK_CUDA_TRY(h, cudaStreamSynchronize(st));
    DeviceFlags fl;
    JK_CUDA_TRY(h, cudaMemcpy(&fl, h->flags, sizeof fl, cudaMemcpyDeviceToHost));
    if (fl.error != 0) {
        JK_CUDA_TRY(h, cudaMemset(h->flags, 0, sizeof(DeviceFlags)));
        return set_error(h, (jk_status)fl.error, "device reported status %d (detail %d)",
                         fl.error, fl.where);
    }
    return JK_OK;
}

const char *jk_status_string(jk_status s) {
    switch (s) {
        case JK_OK: return "ok";
        case JK_ERR_ARG: return "invalid argument";
        case JK_ERR_SHAPE: return "invalid shape";
        case JK_ERR_OOM: return "workspace arena too small";
        case JK_ERR_CUDA: return "CUDA error";
        case JK_ERR_TIMEOUT: return "device wait timed out";
        case JK_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *jk_last_error(jk_handle h) { return h ? h->last_error.c_str() : ""; }

const char *jk_version(void) { return "jk-b300 0.1 (sm_103a)"; }

}  // extern "C"
