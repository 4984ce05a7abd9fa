// C ABI of libjk.so: handle, arena, validation and dispatch (see include/jk.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "jk_internal.h"
#include "packed.cuh"

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
static bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

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
    pb.packed = h && h->packed_factor;
    pb.jpath = h ? h->jpath : -1;
    int c = 0, ks = 0, km = 0;
    for (int s = 0; s < nd; s++) {
        if (d[s].k < 1 || d[s].k > f->nbf * 4)
            return set_error(h, JK_ERR_SHAPE, "density %d: k=%d out of range [1, 4*nbf]", s, d[s].k);
        if (static_cast<long long>(f->nbf) * d[s].k > INT32_MAX)
            return set_error(h, JK_ERR_SHAPE, "density %d: nbf*k=%lld exceeds 2^31-1", s,
                             static_cast<long long>(f->nbf) * d[s].k);
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

// Every device-factor call takes a packed factor (JK_OPT_PACKED_FACTOR); the
// host builds, whose factor lives in host memory, refuse the option.
static jk_status refuse_packed(jk_ctx *h, const char *what) {
    if (h && h->packed_factor)
        return set_error(h, JK_ERR_UNSUPPORTED, "%s does not take a packed factor (JK_OPT_PACKED_FACTOR)", what);
    return JK_OK;
}

// Effective run-time configuration of a call: the tuned entry of its shape
// bucket (when allowed), overridden by options set explicitly on the handle.
static jk_tune_config resolve_config(const jk_ctx *h, jk_op op, jk_precision p, int sms, int nmol,
                                     const Problem *pbs) {
    jk_tune_config c{0, 0, 0};
    if (!h || h->use_tuned) {
        jk_tune_config t;
        if (tune_lookup(tune_key(op, p, sms, nmol, pbs), t)) c = t;
    }
    if (h) {
        if (h->aux_chunk >= 0) c.aux_chunk = h->aux_chunk;
        if (h->schedule >= 0) c.schedule = h->schedule;
        if (h->raster >= 0) c.raster = h->raster;
        if (h->tile >= 0) c.tile = h->tile;
    }
    return c;
}

static void apply_config(Problem &pb, const jk_tune_config &c) {
    pb.aux_chunk = c.aux_chunk;
    pb.schedule = c.schedule;
}

static int current_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms;
}

static jk_status check_out(jk_ctx *h, const void *p, const char *what) {
    if (!p) return JK_OK;
    if (!aligned8(p)) return set_error(h, JK_ERR_ARG, "%s is not 8-byte aligned", what);
    if (!device_readable(p)) return set_error(h, JK_ERR_ARG, "%s is not device memory", what);
    return JK_OK;
}

static jk_status check_in(jk_ctx *h, const void *p, const char *what) {
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
    if (p == JK_FP64) return fp64_build_workspace(pb, fp64_default_pchunk(pb));
    return pb.schedule == 1 ? split_batched_workspace(1, &pb) : split_build_workspace(pb);
}

static size_t batched_bytes(int nmol, const Problem *pbs, jk_precision p) {
    if (p == JK_SPLIT_BF16) return split_batched_workspace(nmol, pbs);
    size_t need = 0;
    for (int m = 0; m < nmol; m++) need = std::max(need, build_bytes(pbs[m], p));
    return need;
}

static jk_status run_build(jk_ctx *h, const Problem &pb, jk_precision p, cudaStream_t st) {
    h->arena.reset(flags_bytes());
    if (p == JK_FP64) return fp64_build(h, pb, st);
    return pb.schedule == 1 ? split_batched(h, 1, &pb, st) : split_build(h, pb, st);
}

static size_t adjoint_bytes(const Problem &pb, jk_precision p, bool want_dl) {
    return p == JK_FP64 ? fp64_adjoint_workspace(pb, fp64_default_pchunk(pb), want_dl)
                        : split_adjoint_workspace(pb, want_dl);
}

// ---- host-resident inputs (jk_build_host) ----------------------------------
// The factor streams to the device in chunks of aux indices; each chunk is an
// ordinary build over its P-range (J and K are sums over P), summed on the
// device in FP64 in chunk order.

static int host_chunk_of(const jk_ctx *h, const Problem &pb) {
    long long c = h && h->host_chunk > 0 ? h->host_chunk : (pb.naux + 11) / 12;
    if (c < 16) c = 16;
    if (c > pb.naux) c = pb.naux;
    return static_cast<int>(c);
}

// Device buffers of a host build that live across its chunks.
struct HostBufs {
    double *XY = nullptr;          // X_s (and Y_s) packed density by density
    double *J = nullptr, *K = nullptr, *Jc = nullptr, *Kc = nullptr;
    double *stage[2] = {nullptr, nullptr};
    double *pstage[2] = {nullptr, nullptr};   // packed factor chunks as uploaded (packed builds)
};

// Doubles of one packed L^P (upper triangle, diagonal included).
using packed::tri_count;

static size_t host_xy_count(const Problem &pb) {
    size_t c = 0;
    for (int s = 0; s < pb.nd; s++) c += static_cast<size_t>(pb.n) * pb.k[s] * (pb.sym[s] ? 1 : 2);
    return c;
}

static size_t host_persist_bytes(const Problem &pb, int chunk, bool wantJ, bool wantK, bool packed = false) {
    const size_t nn = static_cast<size_t>(pb.nd) * pb.n * pb.n * 8;
    return align_up(host_xy_count(pb) * 8) + (wantJ ? 2 * align_up(nn) : 0) + (wantK ? 2 * align_up(nn) : 0) +
           2 * align_up(static_cast<size_t>(chunk) * pb.n * pb.n * 8) +
           (packed ? 2 * align_up(static_cast<size_t>(chunk) * tri_count(pb.n) * 8) : 0) + 8 * kArenaAlign;
}

// The per-chunk problem: device copies of the densities, a staging factor.
static Problem host_chunk_problem(const Problem &pb, const HostBufs &b, int np, int buf) {
    Problem q = pb;
    q.naux = np;
    if (q.jpath < 0) q.jpath = j_on_tensor(pb) ? 1 : 0;   // J's form chosen for the whole problem
    q.L = b.stage[buf];
    size_t off = 0;
    for (int s = 0; s < pb.nd; s++) {
        const size_t cnt = static_cast<size_t>(pb.n) * pb.k[s];
        q.X[s] = b.XY + off;
        off += cnt;
        if (pb.sym[s]) {
            q.Y[s] = q.X[s];
        } else {
            q.Y[s] = b.XY + off;
            off += cnt;
        }
    }
    const long long n2 = static_cast<long long>(pb.n) * pb.n;
    for (int s = 0; s < pb.nd; s++) {
        q.J[s] = pb.wantJ ? b.Jc + s * n2 : nullptr;
        q.K[s] = pb.wantK ? b.Kc + s * n2 : nullptr;
    }
    return q;
}

// Configuration of the chunk builds: tuned for the chunk shape, else the
// grouped schedule (one launch per phase for all densities of the chunk).
static jk_tune_config host_config(const jk_ctx *h, jk_precision p, const Problem &q) {
    jk_tune_config c{0, 1, 0};
    jk_tune_config t;
    if (h->use_tuned && tune_lookup(tune_key(JK_OP_BUILD, p, h->num_sms, 1, &q), t)) c = t;
    if (h->aux_chunk >= 0) c.aux_chunk = h->aux_chunk;
    if (h->schedule >= 0) c.schedule = h->schedule;
    if (h->raster >= 0) c.raster = h->raster;
    if (h->tile >= 0) c.tile = h->tile;
    return c;
}

static size_t host_build_bytes(const jk_ctx *h, const Problem &pb, jk_precision p, bool packed = false) {
    const int chunk = host_chunk_of(h, pb);
    Problem q = pb;
    q.naux = chunk;
    if (q.jpath < 0) q.jpath = j_on_tensor(pb) ? 1 : 0;   // as the chunk builds take it
    jk_tune_config c{0, 1, 0};
    if (h) c = host_config(h, p, q);
    apply_config(q, c);
    return host_persist_bytes(pb, chunk, true, true, packed) + build_bytes(q, p);
}

static jk_status ensure_copy_stream(jk_ctx *h) {
    if (h->copy_stream) return JK_OK;
    JK_CUDA_TRY(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    JK_CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    for (int i = 0; i < 2; i++) {
        JK_CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_up[i], cudaEventDisableTiming));
        JK_CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_used[i], cudaEventDisableTiming));
    }
    return JK_OK;
}

// With `packed`, pb.L holds each L^P as its packed upper triangle: half the
// bytes are uploaded, and each chunk is expanded on the device before its build.
static jk_status host_build(jk_ctx *h, const Problem &pb, const jk_density *d, double *J, double *K,
                            jk_precision p, cudaStream_t st, bool packed = false) {
    const int n = pb.n, naux = pb.naux, nd = pb.nd;
    const long long n2 = static_cast<long long>(n) * n;
    const size_t nn = static_cast<size_t>(nd) * n2;
    const int chunk = host_chunk_of(h, pb);
    Arena &ar = h->arena;
    HostBufs b;
    b.XY = ar.take<double>(host_xy_count(pb));
    bool ok = b.XY != nullptr;
    if (pb.wantJ) {
        b.J = ar.take<double>(nn);
        b.Jc = ar.take<double>(nn);
        ok = ok && b.J && b.Jc;
    }
    if (pb.wantK) {
        b.K = ar.take<double>(nn);
        b.Kc = ar.take<double>(nn);
        ok = ok && b.K && b.Kc;
    }
    for (int i = 0; i < 2; i++) {
        b.stage[i] = ar.take<double>(static_cast<size_t>(chunk) * n2);
        ok = ok && b.stage[i];
        if (packed) {
            b.pstage[i] = ar.take<double>(static_cast<size_t>(chunk) * tri_count(n));
            ok = ok && b.pstage[i];
        }
    }
    if (!ok) return set_error(h, JK_ERR_OOM, "arena too small for the host build's staging buffers");
    Problem q = host_chunk_problem(pb, b, chunk, 0);
    const jk_tune_config cfg = host_config(h, p, q);
    apply_config(q, cfg);
    if (ar.off + build_bytes(q, p) > ar.bytes)
        return set_error(h, JK_ERR_OOM, "arena has %zu bytes, this host build needs %zu", ar.bytes,
                         ar.off + build_bytes(q, p));
    JK_TRY(ensure_copy_stream(h));
    h->cur_raster = cfg.raster;
    h->cur_tile = cfg.tile;

    // densities up, accumulators cleared (on the caller's stream)
    size_t off = 0;
    for (int s = 0; s < nd; s++) {
        const size_t cnt = static_cast<size_t>(n) * pb.k[s];
        JK_CUDA_TRY(h, cudaMemcpyAsync(b.XY + off, d[s].X, cnt * 8, cudaMemcpyHostToDevice, st));
        off += cnt;
        if (!pb.sym[s]) {
            JK_CUDA_TRY(h, cudaMemcpyAsync(b.XY + off, d[s].Y, cnt * 8, cudaMemcpyHostToDevice, st));
            off += cnt;
        }
    }
    if (pb.wantJ) JK_CUDA_TRY(h, cudaMemsetAsync(b.J, 0, nn * 8, st));
    if (pb.wantK) JK_CUDA_TRY(h, cudaMemsetAsync(b.K, 0, nn * 8, st));
    // the copy stream forks from the caller's stream ...
    JK_CUDA_TRY(h, cudaEventRecord(h->ev_fork, st));
    JK_CUDA_TRY(h, cudaStreamWaitEvent(h->copy_stream, h->ev_fork, 0));
    struct FloorGuard {
        Arena &a;
        ~FloorGuard() { a.floor = 0; }
    } guard{ar};
    ar.floor = ar.off;
    int c = 0;
    for (int P0 = 0; P0 < naux; P0 += chunk, c++) {
        const int np = naux - P0 < chunk ? naux - P0 : chunk;
        const int buf = c & 1;
        // ... uploads chunk c once the build of chunk c - 2 has released its buffer ...
        if (c >= 2) JK_CUDA_TRY(h, cudaStreamWaitEvent(h->copy_stream, h->ev_used[buf], 0));
        const long long per = packed ? tri_count(n) : n2;
        JK_CUDA_TRY(h, cudaMemcpyAsync(packed ? b.pstage[buf] : b.stage[buf], pb.L + P0 * per,
                                       static_cast<size_t>(np) * per * 8, cudaMemcpyHostToDevice, h->copy_stream));
        JK_CUDA_TRY(h, cudaEventRecord(h->ev_up[buf], h->copy_stream));
        // ... and every chunk's build waits for its upload (which also joins the streams)
        JK_CUDA_TRY(h, cudaStreamWaitEvent(st, h->ev_up[buf], 0));
        if (packed) JK_TRY(fp64_unpack_sym(h, b.pstage[buf], n, np, b.stage[buf], st));
        Problem qc = host_chunk_problem(pb, b, np, buf);
        apply_config(qc, cfg);
        JK_TRY(run_build(h, qc, p, st));
        if (pb.wantJ) JK_TRY(fp64_axpy(h, b.J, b.Jc, static_cast<long long>(nn), st));
        if (pb.wantK) JK_TRY(fp64_axpy(h, b.K, b.Kc, static_cast<long long>(nn), st));
        JK_CUDA_TRY(h, cudaEventRecord(h->ev_used[buf], st));
    }
    if (pb.wantJ) JK_CUDA_TRY(h, cudaMemcpyAsync(J, b.J, nn * 8, cudaMemcpyDeviceToHost, st));
    if (pb.wantK) JK_CUDA_TRY(h, cudaMemcpyAsync(K, b.K, nn * 8, cudaMemcpyDeviceToHost, st));
    return JK_OK;
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
    if (!h) return JK_OK;
    if (h->aux_stream) {
        cudaStreamSynchronize(h->aux_stream);
        cudaStreamDestroy(h->aux_stream);
        cudaEventDestroy(h->ev_jfork);
        cudaEventDestroy(h->ev_jdone);
    }
    if (h->copy_stream) {
        cudaStreamSynchronize(h->copy_stream);
        cudaStreamDestroy(h->copy_stream);
        cudaEventDestroy(h->ev_fork);
        for (int i = 0; i < 2; i++) {
            cudaEventDestroy(h->ev_up[i]);
            cudaEventDestroy(h->ev_used[i]);
        }
    }
    delete h;
    return JK_OK;
}

}  // extern "C"

namespace jk {

// Validation shared by jk_build and jk_autotune: the problem and its outputs.
static jk_status prepare_build(jk_ctx *h, const jk_factor *f, int32_t nd, const jk_density *d, double *J,
                               double *K, Problem &pb) {
    JK_TRY(make_problem(h, f, nd, d, true, pb));
    JK_TRY(check_out(h, J, "J"));
    JK_TRY(check_out(h, K, "K"));
    const long long n2 = (long long)pb.n * pb.n;
    pb.wantJ = J != nullptr;
    pb.wantK = K != nullptr;
    for (int s = 0; s < nd; s++) {
        pb.J[s] = J ? J + s * n2 : nullptr;
        pb.K[s] = K ? K + s * n2 : nullptr;
    }
    return JK_OK;
}

// Validation shared by jk_build_batched and jk_autotune_batched.
static jk_status prepare_batched(jk_ctx *h, int32_t nmol, const jk_factor *f, const int32_t *nd_per_mol,
                                 const jk_density *d, double *const *J, double *const *K,
                                 std::vector<Problem> &pbs) {
    if (nmol < 1 || !f || !nd_per_mol || !d)
        return set_error(h, JK_ERR_SHAPE, "nmol=%d or a NULL array", nmol);
    pbs.resize(nmol);
    int off = 0;
    for (int m = 0; m < nmol; m++) {
        Problem &pb = pbs[m];
        JK_TRY(make_problem(h, &f[m], nd_per_mol[m], d + off, true, pb));
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
        off += nd_per_mol[m];
    }
    return JK_OK;
}

// Times each candidate configuration (one warm-up build, then reps builds
// between two events on the stream) and keeps the fastest.  A device error
// flag raised by any candidate ends the search with that status.
template <class Fits, class Run>
static jk_status time_candidates(jk_ctx *h, const std::vector<jk_tune_config> &cands, int reps, cudaStream_t st,
                                 Fits fits, Run run, jk_tune_config &best, double &best_ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    JK_CUDA_TRY(h, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(h, JK_ERR_CUDA, "cudaEventCreate failed");
    }
    jk_status rc = JK_OK;
    bool any = false;
    best_ms = INFINITY;
    for (const auto &c : cands) {
        if (!fits(c)) continue;
        if ((rc = run(c)) != JK_OK) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = set_error(h, JK_ERR_CUDA, "event record failed"); break; }
        for (int r = 0; r < reps && rc == JK_OK; r++) rc = run(c);
        if (rc != JK_OK) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = set_error(h, JK_ERR_CUDA, "event timing failed: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        DeviceFlags fl;
        if (cudaMemcpy(&fl, h->flags, sizeof fl, cudaMemcpyDeviceToHost) != cudaSuccess) {
            rc = set_error(h, JK_ERR_CUDA, "reading the device flags failed");
            break;
        }
        if (fl.error != 0) {
            cudaMemset(h->flags, 0, sizeof(DeviceFlags));
            rc = set_error(h, static_cast<jk_status>(fl.error), "device reported status %d while tuning", fl.error);
            break;
        }
        const double per = ms / reps;
        if (per < best_ms) {
            best_ms = per;
            best = c;
        }
        any = true;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != JK_OK) return rc;
    if (!any) return set_error(h, JK_ERR_OOM, "no candidate configuration fits the arena");
    return JK_OK;
}

// Aux-chunk candidates around the automatic choice pc0 (0 = automatic),
// deduplicated by the chunk they produce.
static std::vector<int> chunk_candidates(int pc0, int naux_max) {
    std::vector<int> out{0};
    std::vector<int> seen{std::min(pc0, naux_max)};
    for (int v : {2 * pc0, pc0 / 2, pc0 / 4}) {
        if (v < 1) continue;
        const int eff = std::min(v, naux_max);
        if (std::find(seen.begin(), seen.end(), eff) != seen.end()) continue;
        seen.push_back(eff);
        out.push_back(v);
    }
    return out;
}

// ---- bra-ket pairings (jk_pair) ---------------------------------------------
// The right densities' J_b and K_b (an ordinary build into workspace buffers
// that outlive it), the packed left factors, then the FP64 contraction
// <A_a B_a^T, M_b> per pair.

static size_t pair_persist_bytes(const Problem &pl, int nr, bool wantJ, bool wantK) {
    const size_t nn = static_cast<size_t>(nr) * pl.n * pl.n * 8;
    return (wantJ ? align_up(nn) : 0) + (wantK ? align_up(nn) : 0) +
           align_up(static_cast<size_t>(pl.n) * pl.ctot * 8) +
           align_up(static_cast<size_t>(nr) * pl.n * pl.ctot * 8) + kArenaAlign;
}

static size_t pair_bytes(const Problem &pl, const Problem &pr, jk_precision p, bool wantJ, bool wantK) {
    return pair_persist_bytes(pl, pr.nd, wantJ, wantK) + build_bytes(pr, p);
}

// ---- Laplace (LT-AO) builds (jk_build_laplace) -------------------------------
// The energy-scaled coefficients of every quadrature point go into workspace
// buffers kept across the build (the arena floor); the nq points are the nq
// densities of one ordinary build.  With weights, each point's J and K land
// in the workspace and a fixed-order weighted sum writes the outputs.

// Densities of the build over the scaled coefficients XY (point k: X_k at
// XY + k*n*m, Y_k at XY + (nq + k)*n*m unless symmetric); with XY NULL only
// the shapes are filled in (for validation and queries).
static void laplace_densities(int n, int nq, int m, bool sym, double *XY, jk_density *d) {
    const size_t nm = static_cast<size_t>(n) * m;
    for (int k = 0; k < nq; k++) {
        d[k].k = m;
        d[k].symmetric = sym ? 1 : 0;
        d[k].X = XY ? XY + k * nm : nullptr;
        d[k].Y = XY && !sym ? XY + (nq + k) * nm : nullptr;
    }
}

static size_t laplace_persist_bytes(int n, int nq, int m, bool sym, bool weighted, bool wantJ, bool wantK) {
    const size_t nm = static_cast<size_t>(n) * m, nn = static_cast<size_t>(nq) * n * n * 8;
    return align_up(nm * nq * (sym ? 1 : 2) * 8) + (weighted && wantJ ? align_up(nn) : 0) +
           (weighted && wantK ? align_up(nn) : 0) + kArenaAlign;
}

// ---- dense densities (jk_build_dense, jk_density_grad) ----------------------

// Shape of a dense call; with check_ptrs, the factor is also checked (the
// arrays are checked by the entry points).
static jk_status make_dense(jk_ctx *h, const jk_factor *f, int32_t nd, bool check_ptrs, DenseProb &dp) {
    if (!f) return set_error(h, JK_ERR_ARG, "factor is NULL");
    if (f->nbf < 1 || f->naux < 1)
        return set_error(h, JK_ERR_SHAPE, "nbf=%d naux=%d must be >= 1", f->nbf, f->naux);
    if (f->nbf > 65535) return set_error(h, JK_ERR_SHAPE, "nbf=%d exceeds 65535", f->nbf);
    if (nd < 1 || nd > kMaxDens) return set_error(h, JK_ERR_SHAPE, "nd=%d must be in [1, %d]", nd, kMaxDens);
    dp.n = f->nbf;
    dp.naux = f->naux;
    dp.nd = nd;
    dp.L = f->L;
    dp.packed = h && h->packed_factor;
    if (check_ptrs) {
        if (!f->L) return set_error(h, JK_ERR_ARG, "factor L is NULL");
        if (!aligned16(f->L)) return set_error(h, JK_ERR_ARG, "factor L is not 16-byte aligned");
        if (!device_readable(f->L)) return set_error(h, JK_ERR_ARG, "factor L is not device memory");
    }
    return JK_OK;
}

static size_t dense_bytes(const DenseProb &dp, jk_precision p) {
    return p == JK_FP64 ? fp64_dense_workspace(dp) : split_dense_workspace(dp);
}

// Workspace of the largest form of a dense call (both maps; for the gradient,
// J formed apart and added), for the query: the pointers only mark presence.
static size_t dense_query_bytes(DenseProb dp, jk_op op, jk_precision p) {
    static const double kShapeOnly = 0.0;
    dp.DK = dp.DJ = &kShapeOnly;
    dp.add_j = op == JK_OP_DENSITY_GRAD;
    return dense_bytes(dp, p);
}

// Run-time configuration of a dense call: the handle's explicit options.
static void dense_config(jk_ctx *h, DenseProb &dp) {
    dp.aux_chunk = h->aux_chunk > 0 ? h->aux_chunk : 0;
    h->cur_raster = h->raster >= 0 ? h->raster : 0;
    h->cur_tile = h->tile >= 0 ? h->tile : 0;
}

static jk_status run_dense(jk_ctx *h, const DenseProb &dp, jk_precision p, cudaStream_t st) {
    const size_t need = flags_bytes() + dense_bytes(dp, p);
    if (h->arena.bytes < need)
        return set_error(h, JK_ERR_OOM, "arena has %zu bytes, this dense call needs %zu", h->arena.bytes, need);
    h->arena.reset(flags_bytes());
    return p == JK_FP64 ? fp64_dense(h, dp, st) : split_dense(h, dp, st);
}

// Problems of a host-only batched call (query, lookup): nd_per_mol must split
// the nd densities of d exactly, and d is never read past its nd entries.
// With one_factor every group uses f[0] (the two sides of a pairing).
static jk_status host_batched_problems(int32_t nmol, const jk_factor *f, const int32_t *nd_per_mol, int32_t nd,
                                       const jk_density *d, std::vector<Problem> &pbs, bool one_factor = false) {
    if (nmol < 1 || !nd_per_mol) return JK_ERR_SHAPE;
    pbs.resize(nmol);
    int off = 0;
    for (int m = 0; m < nmol; m++) {
        if (nd_per_mol[m] < 1 || nd_per_mol[m] > nd - off) return JK_ERR_SHAPE;
        JK_TRY(make_problem(nullptr, &f[one_factor ? 0 : m], nd_per_mol[m], d + off, false, pbs[m]));
        off += nd_per_mol[m];
    }
    return off == nd ? JK_OK : JK_ERR_SHAPE;
}

// Workspace of a call under the configuration the handle would use (h may be
// NULL: then the larger of the default and the tuned configuration).
static jk_status query_impl(const jk_ctx *h, jk_op op, int32_t nmol, const jk_factor *f,
                            const int32_t *nd_per_mol, int32_t nd, const jk_density *d, jk_precision p,
                            size_t *bytes) {
    if (!bytes || !f) return JK_ERR_ARG;
    if (p != JK_FP64 && p != JK_SPLIT_BF16) return JK_ERR_ARG;
    // a packed factor (handle option) is taken by the ordinary builds only
    const bool pk = h && h->packed_factor;
    const int jp = h ? h->jpath : -1;   // the split J path (JK_OPT_J_PATH)
    if (pk && (op == JK_OP_BUILD_HOST || op == JK_OP_BUILD_HOST_PACKED))
        return JK_ERR_UNSUPPORTED;
    if (op == JK_OP_BUILD_DENSE || op == JK_OP_DENSITY_GRAD) {
        DenseProb dp;
        jk_status s = make_dense(nullptr, f, nd, false, dp);
        if (s != JK_OK) return s;
        dp.packed = pk;
        dp.aux_chunk = h && h->aux_chunk > 0 ? h->aux_chunk : 0;
        *bytes = dense_query_bytes(dp, op, p) + flags_bytes() + kArenaAlign;
        return JK_OK;
    }
    if (!d) return JK_ERR_ARG;
    const int sms = h ? h->num_sms : current_sms();
    if (op == JK_OP_LAPLACE) {
        // nd = nq points of width d[0].k, symmetric as d[0]; the weighted form
        if (nd < 1 || nd > kMaxDens) return JK_ERR_SHAPE;
        std::vector<jk_density> dl(nd);
        laplace_densities(f->nbf, nd, d[0].k, d[0].symmetric != 0, nullptr, dl.data());
        Problem pb;
        JK_TRY(make_problem(nullptr, f, nd, dl.data(), false, pb));
        pb.packed = pk;
        pb.jpath = jp;
        Problem q = pb;
        apply_config(pb, resolve_config(h, JK_OP_BUILD, p, sms, 1, &pb));
        apply_config(q, jk_tune_config{0, 0, 0});
        const size_t b = h ? build_bytes(pb, p) : std::max(build_bytes(pb, p), build_bytes(q, p));
        *bytes = b + laplace_persist_bytes(pb.n, nd, d[0].k, d[0].symmetric != 0, true, true, true) +
                 flags_bytes() + kArenaAlign;
        return JK_OK;
    }
    if (op == JK_OP_PAIR) {
        // nmol = 2: nd_per_mol = {left count, right count}, d = left then right
        if (nmol != 2 || !nd_per_mol) return JK_ERR_SHAPE;
        std::vector<Problem> pp;
        JK_TRY(host_batched_problems(2, f, nd_per_mol, nd, d, pp, true));
        for (auto &q : pp) {
            q.packed = pk;
            q.jpath = jp;
        }
        size_t need = 0;
        const jk_tune_config cfgs[2] = {resolve_config(h, JK_OP_BUILD, p, sms, 1, &pp[1]),
                                        jk_tune_config{0, 0, 0}};
        for (int v = 0; v < (h ? 1 : 2); v++) {
            Problem q = pp[1];
            apply_config(q, cfgs[v]);
            need = std::max(need, pair_bytes(pp[0], q, p, true, true));
        }
        *bytes = need + flags_bytes() + kArenaAlign;
        return JK_OK;
    }
    size_t need = 0;
    std::vector<Problem> pbs;
    if (op == JK_OP_BATCHED) {
        JK_TRY(host_batched_problems(nmol, f, nd_per_mol, nd, d, pbs));
        for (auto &q : pbs) {
            q.packed = pk;
            q.jpath = jp;
        }
    } else if (op == JK_OP_BUILD || op == JK_OP_ADJOINT || op == JK_OP_BUILD_HOST || op == JK_OP_BUILD_HOST_PACKED) {
        pbs.resize(1);
        jk_status s = make_problem(nullptr, f, nd, d, false, pbs[0]);
        if (s != JK_OK) return s;
        pbs[0].packed = pk;
        pbs[0].jpath = jp;
        pbs[0].slices = h ? h->adj_slices : 7;   // the split adjoint's operands (the default without a handle)
        nmol = 1;
        if (op == JK_OP_BUILD_HOST || op == JK_OP_BUILD_HOST_PACKED) {
            *bytes = host_build_bytes(h, pbs[0], p, op == JK_OP_BUILD_HOST_PACKED) + flags_bytes() + kArenaAlign;
            return JK_OK;
        }
    } else {
        return JK_ERR_ARG;
    }
    const jk_tune_config cfgs[2] = {resolve_config(h, op, p, sms, nmol, pbs.data()),
                                    jk_tune_config{0, 0, 0}};
    for (int v = 0; v < (h ? 1 : 2); v++) {
        for (auto &pb : pbs) apply_config(pb, cfgs[v]);
        size_t b = op == JK_OP_BATCHED ? batched_bytes(nmol, pbs.data(), p)
                   : op == JK_OP_BUILD ? build_bytes(pbs[0], p)
                                       : adjoint_bytes(pbs[0], p, true);
        need = std::max(need, b);
    }
    *bytes = need + flags_bytes() + kArenaAlign;
    return JK_OK;
}

}  // namespace jk

extern "C" {

jk_status jk_workspace_query(jk_op op, int32_t nmol, const jk_factor *f,
                             const int32_t *nd_per_mol, int32_t nd,
                             const jk_density *d, jk_precision p, size_t *bytes) {
    return query_impl(nullptr, op, nmol, f, nd_per_mol, nd, d, p, bytes);
}

jk_status jk_workspace_query_handle(jk_handle h, jk_op op, int32_t nmol, const jk_factor *f,
                                    const int32_t *nd_per_mol, int32_t nd, const jk_density *d,
                                    jk_precision p, size_t *bytes) {
    if (!h) return JK_ERR_ARG;
    return query_impl(h, op, nmol, f, nd_per_mol, nd, d, p, bytes);
}

jk_status jk_build(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d,
                   double *J, double *K, jk_precision p, void *stream) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    Problem pb;
    JK_TRY(prepare_build(h, f, nd, d, J, K, pb));
    if (!J && !K) return JK_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const jk_tune_config c = resolve_config(h, JK_OP_BUILD, p, h->num_sms, 1, &pb);
    apply_config(pb, c);
    h->cur_raster = c.raster;
    h->cur_tile = c.tile;
    if (h->arena.bytes < flags_bytes() + build_bytes(pb, p))
        return set_error(h, JK_ERR_OOM, "arena has %zu bytes, this build needs %zu",
                         h->arena.bytes, flags_bytes() + build_bytes(pb, p));
    return run_build(h, pb, p, st);
}

static jk_status build_host_impl(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d, double *J,
                                 double *K, jk_precision p, void *stream, bool packed) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    Problem pb;
    JK_TRY(refuse_packed(h, packed ? "jk_build_host_packed" : "jk_build_host"));
    JK_TRY(make_problem(h, f, nd, d, false, pb));
    if (!f->L) return set_error(h, JK_ERR_ARG, "factor L is NULL");
    for (int s = 0; s < nd; s++)
        if (!d[s].X || (!d[s].symmetric && !d[s].Y))
            return set_error(h, JK_ERR_ARG, "density %d: X or Y is NULL", s);
    if (!J && !K) return JK_OK;
    pb.wantJ = J != nullptr;
    pb.wantK = K != nullptr;
    return host_build(h, pb, d, J, K, p, static_cast<cudaStream_t>(stream), packed);
}

jk_status jk_build_host(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d,
                        double *J, double *K, jk_precision p, void *stream) {
    return build_host_impl(h, f, nd, d, J, K, p, stream, false);
}

jk_status jk_build_host_packed(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d,
                               double *J, double *K, jk_precision p, void *stream) {
    return build_host_impl(h, f, nd, d, J, K, p, stream, true);
}

jk_status jk_build_batched(jk_handle h, int32_t nmol, const jk_factor *f,
                           const int32_t *nd_per_mol, const jk_density *d,
                           double *const *J, double *const *K, jk_precision p,
                           void *stream) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Validate everything before launching anything.
    std::vector<Problem> pbs;
    JK_TRY(prepare_batched(h, nmol, f, nd_per_mol, d, J, K, pbs));
    const jk_tune_config c = resolve_config(h, JK_OP_BATCHED, p, h->num_sms, nmol, pbs.data());
    for (auto &pb : pbs) apply_config(pb, c);
    h->cur_raster = c.raster;
    h->cur_tile = c.tile;
    if (h->arena.bytes < flags_bytes() + batched_bytes(nmol, pbs.data(), p))
        return set_error(h, JK_ERR_OOM, "arena has %zu bytes, this batched build needs %zu", h->arena.bytes,
                         flags_bytes() + batched_bytes(nmol, pbs.data(), p));
    if (!J && !K) return JK_OK;
    return batched_build(h, nmol, pbs.data(), p, st);
}

jk_status jk_autotune(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d,
                      double *J, double *K, jk_precision p, void *stream, int32_t reps,
                      jk_tune_config *best, double *best_ms) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    if (reps < 1) return set_error(h, JK_ERR_ARG, "reps=%d must be >= 1", reps);
    Problem pb;
    JK_TRY(prepare_build(h, f, nd, d, J, K, pb));
    if (!J && !K) return set_error(h, JK_ERR_ARG, "J and K are both NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int pc0 = p == JK_FP64 ? [&] { Problem q = pb; q.aux_chunk = 0; return fp64_default_pchunk(q); }()
                                 : split_auto_pchunk(pb);
    std::vector<jk_tune_config> cands;
    for (int ch : chunk_candidates(pc0, pb.naux))
        for (int sc = 0; sc < (p == JK_FP64 ? 1 : 2); sc++)
            for (int ra = 0; ra < (p == JK_FP64 ? 1 : 2); ra++)
                for (int ti = 0; ti < (p == JK_FP64 ? 1 : 2); ti++)
                    cands.push_back(jk_tune_config{ch, sc, ra, ti});
    auto fits = [&](const jk_tune_config &c) {
        Problem q = pb;
        apply_config(q, c);
        return h->arena.bytes >= flags_bytes() + build_bytes(q, p);
    };
    auto run = [&](const jk_tune_config &c) {
        Problem q = pb;
        apply_config(q, c);
        h->cur_raster = c.raster;
        h->cur_tile = c.tile;
        return run_build(h, q, p, st);
    };
    jk_tune_config bc{0, 0, 0};
    double bms = 0.0;
    JK_TRY(time_candidates(h, cands, reps, st, fits, run, bc, bms));
    tune_store(tune_key(JK_OP_BUILD, p, h->num_sms, 1, &pb), bc, bms);
    if (best) *best = bc;
    if (best_ms) *best_ms = bms;
    return JK_OK;
}

jk_status jk_autotune_batched(jk_handle h, int32_t nmol, const jk_factor *f,
                              const int32_t *nd_per_mol, const jk_density *d,
                              double *const *J, double *const *K, jk_precision p,
                              void *stream, int32_t reps, jk_tune_config *best,
                              double *best_ms) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    if (reps < 1) return set_error(h, JK_ERR_ARG, "reps=%d must be >= 1", reps);
    std::vector<Problem> pbs;
    JK_TRY(prepare_batched(h, nmol, f, nd_per_mol, d, J, K, pbs));
    if (!J && !K) return set_error(h, JK_ERR_ARG, "J and K are both NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int pc0 = 1 << 30, naux_max = 0;
    for (auto &pb : pbs) {
        Problem q = pb;
        q.aux_chunk = 0;
        pc0 = std::min(pc0, p == JK_FP64 ? fp64_default_pchunk(q) : split_auto_pchunk(q));
        naux_max = std::max(naux_max, pb.naux);
    }
    std::vector<jk_tune_config> cands;
    for (int ch : chunk_candidates(pc0, naux_max))
        for (int ra = 0; ra < (p == JK_FP64 ? 1 : 2); ra++)
            for (int ti = 0; ti < (p == JK_FP64 ? 1 : 2); ti++)
                cands.push_back(jk_tune_config{ch, 1, ra, ti});
    auto fits = [&](const jk_tune_config &c) {
        std::vector<Problem> q = pbs;
        for (auto &pb : q) apply_config(pb, c);
        return h->arena.bytes >= flags_bytes() + batched_bytes(nmol, q.data(), p);
    };
    auto run = [&](const jk_tune_config &c) {
        std::vector<Problem> q = pbs;
        for (auto &pb : q) apply_config(pb, c);
        h->cur_raster = c.raster;
        h->cur_tile = c.tile;
        return batched_build(h, nmol, q.data(), p, st);
    };
    jk_tune_config bc{0, 1, 0};
    double bms = 0.0;
    JK_TRY(time_candidates(h, cands, reps, st, fits, run, bc, bms));
    tune_store(tune_key(JK_OP_BATCHED, p, h->num_sms, nmol, pbs.data()), bc, bms);
    if (best) *best = bc;
    if (best_ms) *best_ms = bms;
    return JK_OK;
}

jk_status jk_tune_lookup(jk_op op, int32_t nmol, const jk_factor *f, const int32_t *nd_per_mol,
                         int32_t nd, const jk_density *d, jk_precision p, int32_t num_sms,
                         jk_tune_config *cfg) {
    if (!f || !d || !cfg) return JK_ERR_ARG;
    std::vector<Problem> pbs;
    if (op == JK_OP_BATCHED) {
        JK_TRY(host_batched_problems(nmol, f, nd_per_mol, nd, d, pbs));
    } else if (op == JK_OP_BUILD) {
        pbs.resize(1);
        JK_TRY(make_problem(nullptr, f, nd, d, false, pbs[0]));
        nmol = 1;
    } else {
        return JK_ERR_ARG;
    }
    return tune_lookup(tune_key(op, p, num_sms, nmol, pbs.data()), *cfg) ? JK_OK : JK_ERR_UNSUPPORTED;
}

jk_status jk_adjoint(jk_handle h, const jk_factor *f, int32_t nd, const jk_density *d,
                     const double *W, const double *V, double *dX, double *dY,
                     double *dL, jk_precision p, void *stream) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    Problem pb;
    JK_TRY(make_problem(h, f, nd, d, true, pb));
    if (h->aux_chunk >= 0) pb.aux_chunk = h->aux_chunk;
    pb.slices = h->adj_slices;
    h->cur_raster = h->raster >= 0 ? h->raster : 0;
    h->cur_tile = h->tile >= 0 ? h->tile : 0;
    if (!dX || !dY) return set_error(h, JK_ERR_ARG, "dX and dY are required");
    JK_TRY(check_out(h, dX, "dX"));
    JK_TRY(check_out(h, dY, "dY"));
    JK_TRY(check_out(h, dL, "dL"));
    JK_TRY(check_in(h, W, "W"));
    JK_TRY(check_in(h, V, "V"));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    size_t need = flags_bytes() + adjoint_bytes(pb, p, dL != nullptr);
    if (h->arena.bytes < need)
        return set_error(h, JK_ERR_OOM, "arena has %zu bytes, this adjoint needs %zu",
                         h->arena.bytes, need);
    return p == JK_FP64 ? fp64_adjoint(h, pb, W, V, dX, dY, dL, st)
                        : split_adjoint(h, pb, W, V, dX, dY, dL, st);
}

jk_status jk_build_dense(jk_handle h, const jk_factor *f, int32_t nd, const double *D, double *J, double *K,
                         jk_precision p, void *stream) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    DenseProb dp;
    JK_TRY(make_dense(h, f, nd, true, dp));
    if (!D) return set_error(h, JK_ERR_ARG, "D is NULL");
    JK_TRY(check_in(h, D, "D"));
    JK_TRY(check_out(h, J, "J"));
    JK_TRY(check_out(h, K, "K"));
    if (!J && !K) return JK_OK;
    dp.DJ = J ? D : nullptr;
    dp.DK = K ? D : nullptr;
    dp.J = J;
    dp.K = K;
    dense_config(h, dp);
    return run_dense(h, dp, p, static_cast<cudaStream_t>(stream));
}

jk_status jk_density_grad(jk_handle h, const jk_factor *f, int32_t nd, const double *W, const double *V,
                          double *G, jk_precision p, void *stream) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    DenseProb dp;
    JK_TRY(make_dense(h, f, nd, true, dp));
    if (!G) return set_error(h, JK_ERR_ARG, "G is NULL");
    JK_TRY(check_out(h, G, "G"));
    JK_TRY(check_in(h, W, "W"));
    JK_TRY(check_in(h, V, "V"));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!W && !V) {
        // both seeds zero: so is the gradient
        JK_CUDA_TRY(h, cudaMemsetAsync(G, 0, static_cast<size_t>(nd) * dp.n * dp.n * 8, st));
        return JK_OK;
    }
    dp.DK = W;
    dp.DJ = V;
    if (W) {
        dp.K = G;
        dp.add_j = V != nullptr;
    } else {
        dp.J = G;
    }
    dense_config(h, dp);
    return run_dense(h, dp, p, st);
}

jk_status jk_pair(jk_handle h, const jk_factor *f, int32_t nl, const jk_density *left, int32_t nr,
                  const jk_density *right, double *Jp, double *Kp, jk_precision p, void *stream) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    Problem pl, pr;
    JK_TRY(make_problem(h, f, nl, left, true, pl));
    JK_TRY(make_problem(h, f, nr, right, true, pr));
    JK_TRY(check_out(h, Jp, "Jp"));
    JK_TRY(check_out(h, Kp, "Kp"));
    if (!Jp && !Kp) return JK_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const jk_tune_config c = resolve_config(h, JK_OP_BUILD, p, h->num_sms, 1, &pr);
    apply_config(pr, c);
    h->cur_raster = c.raster;
    h->cur_tile = c.tile;
    const size_t need = flags_bytes() + pair_bytes(pl, pr, p, Jp != nullptr, Kp != nullptr);
    if (h->arena.bytes < need)
        return set_error(h, JK_ERR_OOM, "arena has %zu bytes, this pairing needs %zu", h->arena.bytes, need);
    Arena &ar = h->arena;
    const int n = pl.n;
    const size_t nn = static_cast<size_t>(nr) * n * n;
    double *Jall = Jp ? ar.take<double>(nn) : nullptr;
    double *Kall = Kp ? ar.take<double>(nn) : nullptr;
    double *ZL = ar.take<double>(static_cast<size_t>(n) * pl.ctot);
    double *U = ar.take<double>(static_cast<size_t>(nr) * n * pl.ctot);
    if ((Jp && !Jall) || (Kp && !Kall) || !ZL || !U)
        return set_error(h, JK_ERR_OOM, "arena too small for the pairing's buffers");
    const long long n2 = static_cast<long long>(n) * n;
    pr.wantJ = Jp != nullptr;
    pr.wantK = Kp != nullptr;
    for (int b = 0; b < nr; b++) {
        pr.J[b] = Jall ? Jall + b * n2 : nullptr;
        pr.K[b] = Kall ? Kall + b * n2 : nullptr;
    }
    // the right densities' J_b, K_b: an ordinary build above the buffers kept
    struct FloorGuard {
        Arena &a;
        ~FloorGuard() { a.floor = 0; }
    } guard{ar};
    ar.floor = ar.off;
    JK_TRY(run_build(h, pr, p, st));
    JK_TRY(split_pack_z(h, pl, ZL, st));
    if (Jp) JK_TRY(fp64_pair_contract(h, pl, ZL, Jall, nr, U, Jp, st));
    if (Kp) JK_TRY(fp64_pair_contract(h, pl, ZL, Kall, nr, U, Kp, st));
    return JK_OK;
}

jk_status jk_build_laplace(jk_handle h, const jk_factor *f, int32_t nq, const double *alpha, const double *w,
                           int32_t m, const double *CX, const double *epsX, int32_t sx, const double *CY,
                           const double *epsY, int32_t sy, double *J, double *K, jk_precision p, void *stream) {
    JK_TRY(begin_call(h));
    if (p != JK_FP64 && p != JK_SPLIT_BF16)
        return set_error(h, JK_ERR_ARG, "unknown precision %d", (int)p);
    if (!f) return set_error(h, JK_ERR_ARG, "factor is NULL");
    if (nq < 1 || nq > kMaxDens) return set_error(h, JK_ERR_SHAPE, "nq=%d must be in [1, %d]", nq, kMaxDens);
    if (!alpha) return set_error(h, JK_ERR_ARG, "alpha is NULL");
    if (sx != 1 && sx != -1) return set_error(h, JK_ERR_ARG, "sx=%d must be +1 or -1", sx);
    const bool sym = CY == nullptr;
    if (sym != (epsY == nullptr)) return set_error(h, JK_ERR_ARG, "CY and epsY must both be given or both NULL");
    if (!sym && sy != 1 && sy != -1) return set_error(h, JK_ERR_ARG, "sy=%d must be +1 or -1", sy);
    if (!CX || !epsX) return set_error(h, JK_ERR_ARG, "CX or epsX is NULL");
    for (int k = 0; k < nq; k++)
        if (!std::isfinite(alpha[k]) || (w && !std::isfinite(w[k])))
            return set_error(h, JK_ERR_ARG, "alpha[%d] or w[%d] is not finite", k, k);
    JK_TRY(check_in(h, CX, "CX"));
    JK_TRY(check_in(h, epsX, "epsX"));
    JK_TRY(check_in(h, CY, "CY"));
    JK_TRY(check_in(h, epsY, "epsY"));
    JK_TRY(check_out(h, J, "J"));
    JK_TRY(check_out(h, K, "K"));
    // shapes: the nq points are densities of width m over f (as jk_build checks them)
    std::vector<jk_density> d(nq);
    laplace_densities(f->nbf, nq, m, sym, nullptr, d.data());
    Problem pb;
    JK_TRY(make_problem(h, f, nq, d.data(), false, pb));
    if (!f->L) return set_error(h, JK_ERR_ARG, "factor L is NULL");
    if (!aligned16(f->L)) return set_error(h, JK_ERR_ARG, "factor L is not 16-byte aligned");
    if (!device_readable(f->L)) return set_error(h, JK_ERR_ARG, "factor L is not device memory");
    if (!J && !K) return JK_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const jk_tune_config c = resolve_config(h, JK_OP_BUILD, p, h->num_sms, 1, &pb);
    apply_config(pb, c);
    h->cur_raster = c.raster;
    h->cur_tile = c.tile;
    const int n = pb.n;
    const bool weighted = w != nullptr;
    const size_t need = flags_bytes() + laplace_persist_bytes(n, nq, m, sym, weighted, J != nullptr, K != nullptr) +
                        build_bytes(pb, p);
    if (h->arena.bytes < need)
        return set_error(h, JK_ERR_OOM, "arena has %zu bytes, this Laplace build needs %zu", h->arena.bytes, need);
    Arena &ar = h->arena;
    const size_t nm = static_cast<size_t>(n) * m;
    const long long n2 = static_cast<long long>(n) * n;
    double *XY = ar.take<double>(nm * nq * (sym ? 1 : 2));
    double *Jall = weighted && J ? ar.take<double>(static_cast<size_t>(nq) * n2) : nullptr;
    double *Kall = weighted && K ? ar.take<double>(static_cast<size_t>(nq) * n2) : nullptr;
    if (!XY || (weighted && J && !Jall) || (weighted && K && !Kall))
        return set_error(h, JK_ERR_OOM, "arena too small for the Laplace buffers");
    // the scaled coefficients, then the build over them
    JK_TRY(fp64_laplace_scale(h, CX, epsX, n, m, sx, alpha, nq, XY, st));
    if (!sym) JK_TRY(fp64_laplace_scale(h, CY, epsY, n, m, sy, alpha, nq, XY + nq * nm, st));
    laplace_densities(n, nq, m, sym, XY, d.data());
    JK_TRY(make_problem(h, f, nq, d.data(), false, pb));
    apply_config(pb, c);
    pb.wantJ = J != nullptr;
    pb.wantK = K != nullptr;
    for (int k = 0; k < nq; k++) {
        pb.J[k] = J ? (weighted ? Jall : J) + k * n2 : nullptr;
        pb.K[k] = K ? (weighted ? Kall : K) + k * n2 : nullptr;
    }
    struct FloorGuard {
        Arena &a;
        ~FloorGuard() { a.floor = 0; }
    } guard{ar};
    ar.floor = ar.off;
    JK_TRY(run_build(h, pb, p, st));
    if (weighted && J) JK_TRY(fp64_weighted_sum(h, J, Jall, w, nq, n2, st));
    if (weighted && K) JK_TRY(fp64_weighted_sum(h, K, Kall, w, nq, n2, st));
    return JK_OK;
}

jk_status jk_pack_factor(jk_handle h, int32_t nbf, int32_t naux, const double *L, double *P, void *stream) {
    JK_TRY(begin_call(h));
    if (nbf < 1 || nbf > 65535 || naux < 1)
        return set_error(h, JK_ERR_SHAPE, "nbf=%d naux=%d: nbf must be in [1, 65535], naux >= 1", nbf, naux);
    if (!L || !P) return set_error(h, JK_ERR_ARG, "L or P is NULL");
    JK_TRY(check_in(h, L, "L"));
    JK_TRY(check_out(h, P, "P"));
    const long long tri = tri_count(nbf);
    const char *lo = reinterpret_cast<const char *>(L), *po = reinterpret_cast<const char *>(P);
    const long long lb = static_cast<long long>(naux) * nbf * nbf * 8, pb = static_cast<long long>(naux) * tri * 8;
    if (po < lo + lb && lo < po + pb) return set_error(h, JK_ERR_ARG, "L and P overlap");
    return fp64_pack_sym(h, L, nbf, naux, P, static_cast<cudaStream_t>(stream));
}

jk_status jk_set_option(jk_handle h, jk_option opt, int64_t value) {
    if (!h) return JK_ERR_ARG;
    if (opt == JK_OPT_AUX_CHUNK) {
        if (value < -1 || value > (1 << 30)) return set_error(h, JK_ERR_ARG, "aux chunk out of range");
        h->aux_chunk = static_cast<int>(value);
        return JK_OK;
    }
    if (opt == JK_OPT_SCHEDULE || opt == JK_OPT_RASTER) {
        if (value < -1 || value > 1) return set_error(h, JK_ERR_ARG, "option %d takes -1, 0 or 1", (int)opt);
        (opt == JK_OPT_SCHEDULE ? h->schedule : h->raster) = static_cast<int>(value);
        return JK_OK;
    }
    if (opt == JK_OPT_HOST_CHUNK) {
        if (value < 0 || value > (1 << 30)) return set_error(h, JK_ERR_ARG, "host chunk out of range");
        h->host_chunk = static_cast<int>(value);
        return JK_OK;
    }
    if (opt == JK_OPT_SLICER) {
        if (value != 0 && value != 1) return set_error(h, JK_ERR_ARG, "JK_OPT_SLICER takes 0 or 1");
        h->slicer = static_cast<int>(value);
        return JK_OK;
    }
    if (opt == JK_OPT_SYRK) {
        if (value != 0 && value != 1) return set_error(h, JK_ERR_ARG, "JK_OPT_SYRK takes 0 or 1");
        h->syrk = static_cast<int>(value);
        return JK_OK;
    }
    if (opt == JK_OPT_PACKED_FACTOR) {
        if (value != 0 && value != 1) return set_error(h, JK_ERR_ARG, "JK_OPT_PACKED_FACTOR takes 0 or 1");
        h->packed_factor = static_cast<int>(value);
        return JK_OK;
    }
    if (opt == JK_OPT_TILE) {
        if (value < -1 || value > 1) return set_error(h, JK_ERR_ARG, "JK_OPT_TILE takes -1, 0 or 1");
        h->tile = static_cast<int>(value);
        return JK_OK;
    }
    if (opt == JK_OPT_ADJOINT_SLICES) {
        if (value != 6 && value != 7) return set_error(h, JK_ERR_ARG, "JK_OPT_ADJOINT_SLICES takes 6 or 7");
        h->adj_slices = static_cast<int>(value);
        return JK_OK;
    }
    if (opt == JK_OPT_J_PATH) {
        if (value < -1 || value > 1) return set_error(h, JK_ERR_ARG, "JK_OPT_J_PATH takes -1, 0 or 1");
        h->jpath = static_cast<int>(value);
        return JK_OK;
    }
    if (opt == JK_OPT_USE_TUNED) {
        if (value != 0 && value != 1) return set_error(h, JK_ERR_ARG, "JK_OPT_USE_TUNED takes 0 or 1");
        h->use_tuned = static_cast<int>(value);
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
