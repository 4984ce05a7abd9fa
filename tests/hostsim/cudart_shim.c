/*
 * cudart_shim.c -- TEST INFRASTRUCTURE: a stand-in for the CUDA runtime so
 * that libjk.so's host code (validation, workspace arithmetic, the sequence
 * of launches, tensor-map encoding) runs end to end on a machine without a
 * GPU.  Built as libcudart.so.13 and found first on LD_LIBRARY_PATH by a
 * child process; nothing here runs device code.
 *
 *  - "device memory" is host memory: every pointer reports as device memory,
 *    copies and memsets act on host memory;
 *  - kernel launches are recorded (kernel name, grid, block, dynamic shared
 *    memory, cluster shape), not executed;
 *  - cuTensorMapEncodeTiled (through the driver entry point) is recorded
 *    (type, rank, base, extents, strides, box, swizzle) and succeeds;
 *  - streams and events are inert handles; timings read 1 ms.
 * The recorded launches and tensor maps are read back with shim_* calls.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <cuda.h>
#include <cuda_runtime_api.h>

#define MAX_FUNCS 1024
#define MAX_LAUNCH 200000
#define MAX_TMAP 200000
#define MAX_VARS 64

static struct { const void *host; const char *name; } g_funcs[MAX_FUNCS];
static int g_nfuncs;

typedef struct {
    int func;
    unsigned grid[3], block[3], cluster[3];
    size_t smem;
} Launch;
static Launch *g_launch;
static int g_nlaunch;

typedef struct {
    int dtype, rank, swizzle;
    const void *base;
    unsigned long long dims[5], strides[5];
    unsigned box[5];
} TMap;
static TMap *g_tmap;
static int g_ntmap;

static struct { const void *host; size_t size; void *buf; } g_vars[MAX_VARS];
static int g_nvars;

static struct { dim3 grid, block; size_t smem; void *stream; } g_cfg;
static int g_fail_launch;
static int g_fail_at = -1;   /* index (within the current case) of a launch made to fail, or -1 */
static int g_launch_error;   /* a failed launch not yet reported by cudaGetLastError */
static int g_ncopies;   /* memsets and copies enqueued on a stream */
static int g_nsync;     /* calls that wait for the device (illegal while capturing a graph) */
static int g_nsetup;    /* one-time set-up: streams, events, function attributes, symbol and entry lookups */

/* Called at every launch while the argument array is alive, so the test can
 * decode each kernel's arguments from its signature. */
typedef void (*launch_hook_t)(const char *name, const unsigned *grid, const unsigned *block, void **args);
static launch_hook_t g_hook;
void shim_set_hook(launch_hook_t h) { g_hook = h; }

static int func_index(const void *host) {
    for (int i = 0; i < g_nfuncs; i++)
        if (g_funcs[i].host == host) return i;
    return -1;
}

/* Returns nonzero when this launch is the one made to fail (it is then not
 * recorded and the kernel does not "run"). */
static int record_launch(const void *host, dim3 grid, dim3 block, size_t smem, const unsigned *cluster,
                         void **args) {
    if (g_fail_at >= 0 && g_nlaunch == g_fail_at) {
        g_fail_at = -1;
        g_launch_error = 1;
        return 1;
    }
    if (g_hook) {
        const int f = func_index(host);
        const unsigned g[3] = {grid.x, grid.y, grid.z}, b[3] = {block.x, block.y, block.z};
        g_hook(f >= 0 ? g_funcs[f].name : "?", g, b, args);
    }
    if (!g_launch) g_launch = (Launch *)calloc(MAX_LAUNCH, sizeof(Launch));
    if (g_nlaunch >= MAX_LAUNCH) { g_fail_launch = 1; return 0; }
    Launch *l = &g_launch[g_nlaunch++];
    l->func = func_index(host);
    l->grid[0] = grid.x; l->grid[1] = grid.y; l->grid[2] = grid.z;
    l->block[0] = block.x; l->block[1] = block.y; l->block[2] = block.z;
    l->smem = smem;
    for (int i = 0; i < 3; i++) l->cluster[i] = cluster ? cluster[i] : 1;
    return 0;
}

/* ---- module registration and launch hooks -------------------------------- */
void **__cudaRegisterFatBinary(void *fatCubin) { (void)fatCubin; static void *h; return &h; }
void __cudaRegisterFatBinaryEnd(void **h) { (void)h; }
void __cudaUnregisterFatBinary(void **h) { (void)h; }

void __cudaRegisterFunction(void **h, const char *hostFun, char *deviceFun, const char *deviceName, int tl,
                            uint3 *tid, uint3 *bid, dim3 *bDim, dim3 *gDim, int *wSize) {
    (void)h; (void)deviceFun; (void)tl; (void)tid; (void)bid; (void)bDim; (void)gDim; (void)wSize;
    if (g_nfuncs < MAX_FUNCS) {
        g_funcs[g_nfuncs].host = hostFun;
        g_funcs[g_nfuncs].name = deviceName;
        g_nfuncs++;
    }
}

void __cudaRegisterVar(void **h, char *hostVar, char *deviceAddress, const char *deviceName, int ext, size_t size,
                       int constant, int global) {
    (void)h; (void)deviceAddress; (void)deviceName; (void)ext; (void)constant; (void)global;
    if (g_nvars < MAX_VARS) {
        g_vars[g_nvars].host = hostVar;
        g_vars[g_nvars].size = size;
        g_vars[g_nvars].buf = NULL;
        g_nvars++;
    }
}

unsigned __cudaPushCallConfiguration(dim3 grid, dim3 block, size_t smem, struct CUstream_st *stream) {
    g_cfg.grid = grid; g_cfg.block = block; g_cfg.smem = smem; g_cfg.stream = stream;
    return 0;
}

cudaError_t __cudaPopCallConfiguration(dim3 *grid, dim3 *block, size_t *smem, void *stream) {
    *grid = g_cfg.grid; *block = g_cfg.block; *smem = g_cfg.smem;
    *(void **)stream = g_cfg.stream;
    return cudaSuccess;
}

cudaError_t __cudaGetKernel(cudaKernel_t *k, const void *fun) { *k = (cudaKernel_t)fun; return cudaSuccess; }

cudaError_t __cudaLaunchKernel(cudaKernel_t kernel, dim3 grid, dim3 block, void **args, size_t smem,
                               cudaStream_t stream) {
    (void)stream;
    return record_launch((const void *)kernel, grid, block, smem, NULL, args) ? cudaErrorLaunchOutOfResources
                                                                               : cudaSuccess;
}

cudaError_t cudaLaunchKernelExC(const cudaLaunchConfig_t *config, const void *func, void **args) {
    unsigned cl[3] = {1, 1, 1};
    for (unsigned i = 0; i < config->numAttrs; i++)
        if (config->attrs[i].id == cudaLaunchAttributeClusterDimension) {
            cl[0] = config->attrs[i].val.clusterDim.x;
            cl[1] = config->attrs[i].val.clusterDim.y;
            cl[2] = config->attrs[i].val.clusterDim.z;
        }
    if (record_launch(func, config->gridDim, config->blockDim, config->dynamicSmemBytes, cl, args)) {
        g_launch_error = 0;   /* reported by the return value, as the runtime does */
        return cudaErrorLaunchOutOfResources;
    }
    return cudaSuccess;
}

cudaError_t cudaFuncSetAttribute(const void *func, enum cudaFuncAttribute attr, int value) {
    (void)func; (void)attr; (void)value;
    g_nsetup++;
    return cudaSuccess;
}

cudaError_t cudaOccupancyMaxActiveClusters(int *n, const void *func, const cudaLaunchConfig_t *cfg) {
    (void)func; (void)cfg;
    g_nsetup++;
    *n = 74;
    return cudaSuccess;
}

/* ---- device, memory, streams, events -------------------------------------- */
cudaError_t cudaGetDevice(int *d) { *d = 0; return cudaSuccess; }

cudaError_t cudaDeviceGetAttribute(int *v, enum cudaDeviceAttr attr, int dev) {
    (void)dev;
    *v = attr == cudaDevAttrMultiProcessorCount ? 148 : 0;
    return cudaSuccess;
}

cudaError_t cudaPointerGetAttributes(struct cudaPointerAttributes *a, const void *p) {
    memset(a, 0, sizeof *a);
    a->type = cudaMemoryTypeDevice;
    a->devicePointer = (void *)p;
    return cudaSuccess;
}

cudaError_t cudaMemset(void *p, int v, size_t n) { g_nsync++; memset(p, v, n); return cudaSuccess; }
cudaError_t cudaMemsetAsync(void *p, int v, size_t n, cudaStream_t s) {
    (void)s; g_ncopies++; memset(p, v, n); return cudaSuccess;
}
cudaError_t cudaMemcpy(void *d, const void *s, size_t n, enum cudaMemcpyKind k) {
    (void)k; g_nsync++; memmove(d, s, n); return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void *d, const void *s, size_t n, enum cudaMemcpyKind k, cudaStream_t st) {
    (void)k; (void)st; g_ncopies++; memmove(d, s, n); return cudaSuccess;
}

cudaError_t cudaGetSymbolAddress(void **p, const void *symbol) {
    g_nsetup++;
    for (int i = 0; i < g_nvars; i++)
        if (g_vars[i].host == symbol) {
            if (!g_vars[i].buf) g_vars[i].buf = aligned_alloc(256, (g_vars[i].size + 255) / 256 * 256);
            *p = g_vars[i].buf;
            return cudaSuccess;
        }
    return cudaErrorInvalidSymbol;
}

static char g_handles[256];
static int g_nhandles;
static void *new_handle(void) { return &g_handles[(g_nhandles++) % 256]; }

cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned f) { (void)f; g_nsetup++; *s = (cudaStream_t)new_handle(); return cudaSuccess; }
cudaError_t cudaStreamDestroy(cudaStream_t s) { (void)s; return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t s) { (void)s; g_nsync++; return cudaSuccess; }
cudaError_t cudaStreamWaitEvent(cudaStream_t s, cudaEvent_t e, unsigned f) { (void)s; (void)e; (void)f; return cudaSuccess; }
cudaError_t cudaEventCreate(cudaEvent_t *e) { g_nsetup++; *e = (cudaEvent_t)new_handle(); return cudaSuccess; }
cudaError_t cudaEventCreateWithFlags(cudaEvent_t *e, unsigned f) { (void)f; g_nsetup++; *e = (cudaEvent_t)new_handle(); return cudaSuccess; }
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t s) { (void)e; (void)s; return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t e) { (void)e; g_nsync++; return cudaSuccess; }
cudaError_t cudaEventElapsedTime(float *ms, cudaEvent_t a, cudaEvent_t b) { (void)a; (void)b; *ms = 1.0f; return cudaSuccess; }
cudaError_t cudaEventDestroy(cudaEvent_t e) { (void)e; return cudaSuccess; }

cudaError_t cudaGetLastError(void) {
    if (g_launch_error) {
        g_launch_error = 0;
        return cudaErrorLaunchOutOfResources;
    }
    return g_fail_launch ? cudaErrorLaunchFailure : cudaSuccess;
}
const char *cudaGetErrorString(cudaError_t e) { return e == cudaSuccess ? "no error" : "host simulation error"; }

/* ---- tensor maps ------------------------------------------------------------ */
static CUresult encode_tiled(CUtensorMap *map, CUtensorMapDataType dtype, cuuint32_t rank, void *base,
                             const cuuint64_t *dims, const cuuint64_t *strides, const cuuint32_t *box,
                             const cuuint32_t *estr, CUtensorMapInterleave il, CUtensorMapSwizzle sw,
                             CUtensorMapL2promotion l2, CUtensorMapFloatOOBfill oob) {
    (void)estr; (void)il; (void)l2; (void)oob;
    memset(map, 0, sizeof *map);
    /* The map is opaque to the library: record what it addresses in it, so a
     * test executing the kernel can find its operand (magic, type, rank, base,
     * extents, byte strides of dimensions 1 and 2). */
    {
        unsigned long long *w = (unsigned long long *)map;
        w[0] = 0x6A6B73696D6D6170ull;
        w[1] = ((unsigned long long)dtype << 32) | rank;
        w[2] = (unsigned long long)(uintptr_t)base;
        for (unsigned i = 0; i < rank && i < 3; i++) w[3 + i] = dims[i];
        for (unsigned i = 1; i < rank && i < 3; i++) w[5 + i] = strides[i - 1];
    }
    if (!g_tmap) g_tmap = (TMap *)calloc(MAX_TMAP, sizeof(TMap));
    if (g_ntmap >= MAX_TMAP || rank < 1 || rank > 5) return CUDA_ERROR_INVALID_VALUE;
    TMap *t = &g_tmap[g_ntmap++];
    t->dtype = (int)dtype;
    t->rank = (int)rank;
    t->swizzle = (int)sw;
    t->base = base;
    for (unsigned i = 0; i < rank; i++) {
        t->dims[i] = dims[i];
        t->box[i] = box[i];
        t->strides[i] = i == 0 ? 0 : strides[i - 1];
    }
    return CUDA_SUCCESS;
}

cudaError_t cudaGetDriverEntryPointByVersion(const char *symbol, void **fn, unsigned int ver, unsigned long long flags,
                                             enum cudaDriverEntryPointQueryResult *status) {
    (void)ver; (void)flags;
    g_nsetup++;
    if (strcmp(symbol, "cuTensorMapEncodeTiled") == 0) {
        *fn = (void *)encode_tiled;
        if (status) *status = cudaDriverEntryPointSuccess;
        return cudaSuccess;
    }
    *fn = NULL;
    if (status) *status = cudaDriverEntryPointSymbolNotFound;
    return cudaSuccess;
}

/* ---- read-back for the test driver ----------------------------------------- */
int shim_var(int i, void **p, size_t *size) {
    if (i >= g_nvars) return 0;
    *p = g_vars[i].buf;
    *size = g_vars[i].size;
    return 1;
}

void shim_fail_launch_at(int i) { g_fail_at = i; g_launch_error = 0; }
int shim_launch_count(void) { return g_nlaunch; }
int shim_tmap_count(void) { return g_ntmap; }
int shim_copy_count(void) { return g_ncopies; }
int shim_sync_count(void) { return g_nsync; }
int shim_setup_count(void) { return g_nsetup; }
void shim_reset(void) { g_nlaunch = 0; g_ntmap = 0; g_fail_launch = 0; g_ncopies = 0; g_nsync = 0; g_nsetup = 0; }

const char *shim_launch(int i, unsigned *grid, unsigned *block, unsigned *cluster, size_t *smem) {
    const Launch *l = &g_launch[i];
    memcpy(grid, l->grid, sizeof l->grid);
    memcpy(block, l->block, sizeof l->block);
    memcpy(cluster, l->cluster, sizeof l->cluster);
    *smem = l->smem;
    return l->func >= 0 ? g_funcs[l->func].name : "?";
}

void shim_tmap(int i, int *dtype_rank_swizzle, unsigned long long *base, unsigned long long *dims,
               unsigned long long *strides, unsigned *box) {
    const TMap *t = &g_tmap[i];
    dtype_rank_swizzle[0] = t->dtype;
    dtype_rank_swizzle[1] = t->rank;
    dtype_rank_swizzle[2] = t->swizzle;
    *base = (unsigned long long)(uintptr_t)t->base;
    memcpy(dims, t->dims, sizeof t->dims);
    memcpy(strides, t->strides, sizeof t->strides);
    memcpy(box, t->box, sizeof t->box);
}
