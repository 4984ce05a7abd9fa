// jk_build_noalloc: the plain FP64 J/K build for callers that cannot allocate
// device memory.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not
// wanted -- inside a CUDA-graph stream capture (allocation is illegal while
// capturing), in plugins or callbacks of a host application that owns the
// device memory budget and forbids its guests to allocate, or in
// latency-critical loops where an allocation could synchronize the device.
// Such callers still own J, K and the inputs; the only thing this entry point
// takes from them is the need for a workspace arena.
//
// The workspace is a file-scope device array of JK_STATIC_SCRATCH_BYTES that
// lives in every GPU's memory from the moment the library's module is loaded
// on that GPU until the process exits.  Host code must not pass the array's
// name to a kernel (on the host it is only a stand-in symbol); the device
// address is looked up once per device with cudaGetSymbolAddress.
#include <atomic>
#include <mutex>

#include "jk_internal.h"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[JK_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device; looked up on the
// first call for that device.  Returns JK_ERR_CUDA if the lookup fails.
jk_status scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return JK_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return JK_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return JK_OK;
}

}  // namespace

extern "C" jk_status jk_build_noalloc(const jk_factor *f, int32_t nd, const jk_density *d, double *J,
                                      double *K, void *stream) {
    using namespace jk;
    if (!f || !d) return JK_ERR_ARG;
    if (!J && !K) return JK_OK;
    if (f->nbf < 1 || f->nbf > 65535 || f->naux < 1 || nd < 1 || nd > kMaxDens) return JK_ERR_SHAPE;
    if (!f->L || (reinterpret_cast<uintptr_t>(f->L) & 15u)) return JK_ERR_ARG;
    if ((J && (reinterpret_cast<uintptr_t>(J) & 15u)) || (K && (reinterpret_cast<uintptr_t>(K) & 15u)))
        return JK_ERR_ARG;
    // Describe the problem exactly as jk_build does (no pointer attribute
    // queries here: the inputs are taken as device pointers).
    Problem pb;
    pb.n = f->nbf;
    pb.naux = f->naux;
    pb.nd = nd;
    pb.L = f->L;
    int c = 0, kmax = 0, ksum = 0;
    for (int s = 0; s < nd; s++) {
        if (d[s].k < 1 || d[s].k > f->nbf * 4 || static_cast<long long>(f->nbf) * d[s].k > INT32_MAX)
            return JK_ERR_SHAPE;
        if (!d[s].X || (!d[s].symmetric && !d[s].Y)) return JK_ERR_ARG;
        if ((reinterpret_cast<uintptr_t>(d[s].X) & 15u) ||
            (!d[s].symmetric && (reinterpret_cast<uintptr_t>(d[s].Y) & 15u)))
            return JK_ERR_ARG;
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
        ksum += d[s].k;
        if (d[s].k > kmax) kmax = d[s].k;
    }
    pb.ctot = c;
    pb.ksum = ksum;
    pb.kmax = kmax;
    const size_t head = align_up(sizeof(DeviceFlags));
    const size_t need = head + fp64_build_workspace(pb, fp64_default_pchunk(pb));
    if (need > JK_STATIC_SCRATCH_BYTES) return JK_ERR_OOM;   // problem too large for the static scratch
    const long long n2 = static_cast<long long>(pb.n) * pb.n;
    pb.wantJ = J != nullptr;
    pb.wantK = K != nullptr;
    for (int s = 0; s < nd; s++) {
        pb.J[s] = J ? J + s * n2 : nullptr;
        pb.K[s] = K ? K + s * n2 : nullptr;
    }
    void *base = nullptr;
    jk_status st = scratch_address(&base);
    if (st != JK_OK) return st;
    // A call-local context over the static scratch.  The FP64 build writes
    // every workspace word before reading it, so only the status words at
    // the start are cleared.
    jk_ctx ctx;
    ctx.arena.base = static_cast<char *>(base);
    ctx.arena.bytes = JK_STATIC_SCRATCH_BYTES;
    ctx.flags = reinterpret_cast<DeviceFlags *>(base);
    ctx.arena.reset(head);
    cudaGetDevice(&ctx.device);
    cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, ctx.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(base, 0, sizeof(DeviceFlags), s) != cudaSuccess) {
        cudaGetLastError();
        return JK_ERR_CUDA;
    }
    return fp64_build(&ctx, pb, s);
}
