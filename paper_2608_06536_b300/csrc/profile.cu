// Launch accounting and per-kernel-kind CUDA-event timing.
#include "jk_internal.h"

namespace jk {

static const char *kKindNames[KK_COUNT] = {
    "dgemm_fp64", "jstream_fp64", "frob_stream_fp64", "gamma_panel_fp64", "pack",
    "misc", "slice", "ozgemm_tcgen05", "oz_reduce", "expo", "j_tri"};

static cudaEvent_t take_event(Profiler &p) {
    if (p.used == p.pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        p.pool.push_back(e);
    }
    return p.pool[p.used++];
}

LaunchScope::LaunchScope(jk_ctx *h_, int kind_, cudaStream_t st_) : h(h_), kind(kind_), st(st_) {
    h->prof.launches++;
    if (!h->prof.on) return;
    cudaEvent_t a = take_event(h->prof);
    b = take_event(h->prof);
    if (!a || !b) { b = nullptr; return; }
    cudaEventRecord(a, st);
    h->prof.recs.push_back({kind, a, b});
}

LaunchScope::~LaunchScope() {
    if (b) cudaEventRecord(b, st);
}

static void drain(jk_ctx *h) {
    Profiler &p = h->prof;
    for (auto &r : p.recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            p.ms[r.kind] += ms;
            p.cnt[r.kind] += 1;
        }
        cudaGetLastError();
    }
    p.recs.clear();
    p.used = 0;
}

// Sixteen independent FMA chains per thread, the loop unrolled four times:
// the FP64 pipe's issue rate with no memory traffic and almost no other
// instructions.  The result is stored only if it equals a value the chains
// cannot reach, which keeps them live without a store per thread.
__global__ void __launch_bounds__(256) fma_stream_kernel(int iters, double *sink) {
    double a[16];
#pragma unroll
    for (int j = 0; j < 16; j++) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
    const double b = 0.999999, c = 1e-7;
#pragma unroll 4
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 16; j++) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 16; j++) s += a[j];
    if (s == -1.0) *sink = s;
}

}  // namespace jk

using namespace jk;

extern "C" {

int64_t jk_launch_count(jk_handle h) { return h ? h->prof.launches : 0; }

jk_status jk_profile_enable(jk_handle h, int32_t on) {
    if (!h) return JK_ERR_ARG;
    h->prof.on = on != 0;
    return JK_OK;
}

jk_status jk_profile_reset(jk_handle h) {
    if (!h) return JK_ERR_ARG;
    drain(h);
    h->prof.launches = 0;
    h->prof.tensor_flops = 0.0;
    for (int i = 0; i < KK_COUNT; i++) { h->prof.ms[i] = 0; h->prof.cnt[i] = 0; }
    return JK_OK;
}

double jk_issued_tensor_flops(jk_handle h) { return h ? h->prof.tensor_flops : 0.0; }

int32_t jk_profile_kinds(void) { return KK_COUNT; }

const char *jk_profile_kind_name(int32_t kind) {
    return (kind >= 0 && kind < KK_COUNT) ? kKindNames[kind] : nullptr;
}

jk_status jk_profile_read(jk_handle h, int32_t kind, double *ms, int64_t *launches) {
    if (!h || kind < 0 || kind >= KK_COUNT) return JK_ERR_ARG;
    drain(h);
    if (ms) *ms = h->prof.ms[kind];
    if (launches) *launches = h->prof.cnt[kind];
    return JK_OK;
}

jk_status jk_debug_fp64_fma(jk_handle h, int32_t blocks_per_sm, int32_t iters, double *sink, double *flops,
                            void *stream) {
    if (!h || !sink || !flops) return JK_ERR_ARG;
    if (blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || iters > (1 << 24))
        return set_error(h, JK_ERR_ARG, "blocks_per_sm must be in [1, 64] and iters in [1, 2^24]");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int grid = blocks_per_sm * h->num_sms;
    {
        LaunchScope ls(h, KK_MISC, st);
        fma_stream_kernel<<<grid, 256, 0, st>>>(iters, sink);
    }
    JK_LAUNCH_CHECK(h);
    *flops = 2.0 * 16.0 * static_cast<double>(iters) * grid * 256.0;
    return JK_OK;
}

}  // extern "C"
