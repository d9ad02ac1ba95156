// wp_probe_accumulate_static: the probe contraction of wp_probe_accumulate for callers
// that cannot give the library any device scratch memory.
//
// Some callers only hold device pointers to their own inputs and outputs and are not
// allowed to allocate more: for example a plug-in running inside a host application whose
// framework owns the whole device through its own allocator, or a serving process whose
// memory budget was fixed when it started.  For them the scratch this call needs (the
// bfloat16 hi/lo copy of the probing matrix and the device error flag) lives in a
// file-scope device array of fixed size, reserved on every GPU that loads the library
// until the process exits.  Nothing here calls cudaMalloc, cudaFree or any allocating
// library routine.
#include <cuda.h>

#include <mutex>

#include "wp_internal.cuh"

namespace {

// Fixed scratch: 16 MiB on every device that loads libwp.so.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device ordinal.  In host code the array's name
// is only a host-side stand-in, so the real address is looked up with
// cudaGetSymbolAddress while that device is current: once per device and context.  The
// context's unique id is kept beside the address, so that after a cudaDeviceReset (a new
// primary context, in which the array may sit elsewhere) the next call looks it up again.
constexpr int kMaxDevices = 64;
void *g_static_ptr[kMaxDevices] = {};
unsigned long long g_static_ctx[kMaxDevices] = {};
std::mutex g_static_mtx;

typedef CUresult (*ctx_current_fn)(CUcontext *);
typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0 if it cannot be read).
unsigned long long current_context_id()
{
    static ctx_current_fn get_current = nullptr;
    static ctx_id_fn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (ctx_current_fn)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (ctx_id_fn)p;
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// Device address of the array on the current device (set-up on first use per context).
cudaError_t static_base(void **base)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    // Before the runtime's first call on this thread no context may be current (id 0):
    // cudaGetSymbolAddress makes the device's primary context current, and the id read
    // after it is the one the call's kernels run in.
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_static_mtx);
    if (!g_static_ptr[dev] || ctx == 0 || ctx != g_static_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
        g_static_ptr[dev] = p;
        g_static_ctx[dev] = current_context_id();
    }
    *base = g_static_ptr[dev];
    return cudaSuccess;
}

// Failures are reported through wp_last_error() like every other call.
wp_status static_fail(wp_status st, const char *msg, cudaError_t e = cudaSuccess)
{
    std::string m = msg;
    if (e != cudaSuccess) {
        m += ": ";
        m += cudaGetErrorString(e);
    }
    wp::set_last_error(m.c_str());
    return st;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" wp_status wp_probe_accumulate_static(const float *A, int cnt, long long npoints,
                                                int nshots, const float *Q, int nt, int t0,
                                                int r, float scale, float *P, wp_stream stream)
{
    if (!A || !Q || !P) return static_fail(WP_ERR_INVALID, "A, Q and P are required");
    if (cnt < 1 || npoints < 1 || nshots < 1 || r < 1 || r > 256 || nt < 1 || t0 < 0 ||
        t0 + cnt > nt || t0 % 8)
        return static_fail(WP_ERR_INVALID,
                           "need 1 <= r <= 256, 0 <= t0, t0 % 8 == 0, t0 + cnt <= nt");
    if (((uintptr_t)A & 15) || ((uintptr_t)Q & 15) || ((uintptr_t)P & 15))
        return static_fail(WP_ERR_INVALID, "device pointers must be 16-byte aligned");
    const int r_pad = r < 16 ? 16 : (r + 15) / 16 * 16;
    const int nt_pad = (nt + 63) / 64 * 64 + 64;
    const size_t q_bytes = (size_t)nshots * r_pad * nt_pad * sizeof(__nv_bfloat16);
    const size_t need = 256 + round256(q_bytes) + q_bytes;
    if (need > kStaticScratchBytes)
        return static_fail(WP_ERR_OOM,
                           "nshots * r_pad * (nt_pad) * 4 bytes exceeds the 16 MiB static "
                           "scratch of wp_probe_accumulate_static");
    void *base = nullptr;
    cudaError_t e = static_base(&base);
    if (e != cudaSuccess)
        return static_fail(WP_ERR_CUDA, "looking up the static scratch (cudaGetSymbolAddress) failed", e);
    cudaStream_t s = (cudaStream_t)stream;
    char *b = (char *)base;
    int *err = (int *)b;
    __nv_bfloat16 *qhi = (__nv_bfloat16 *)(b + 256);
    __nv_bfloat16 *qlo = (__nv_bfloat16 *)(b + 256 + round256(q_bytes));
    // The array keeps the previous call's contents: the error flag must start at zero.
    e = cudaMemsetAsync(err, 0, 256, s);
    if (e != cudaSuccess) return static_fail(WP_ERR_CUDA, "clearing the error flag failed", e);
    e = wp::launch_probe_split(Q, nshots, nt, r, r_pad, nt_pad, qhi, qlo, s);
    if (e != cudaSuccess) return static_fail(WP_ERR_CUDA, "probe split launch failed", e);
    wp::GemmArgs G{};
    G.ring = A;
    G.ring_ss = (long long)cnt * npoints;
    G.nslots = cnt;
    G.N = npoints;
    G.t0 = t0;
    G.cnt = cnt;
    G.slot0 = 0;
    G.mode = 0;
    G.qhi = qhi;
    G.qlo = qlo;
    G.q_ss = (long long)r_pad * nt_pad;
    G.nt_pad = nt_pad;
    G.r = r;
    G.r_pad = r_pad;
    G.P = P;
    G.P_ss = (long long)r * npoints;
    G.scale = scale;
    G.err = err;
    e = wp::launch_probe_gemm(G, nshots, s);
    if (e != cudaSuccess) return static_fail(WP_ERR_CUDA, "probe contraction launch failed", e);
    return WP_OK;
}

// Status of the last wp_probe_accumulate_static call on the current device: polls `stream`
// from the host with a deadline (never spinning on the device), then reads the error flag
// at the start of the static array with a plain device-to-host copy (no allocation).
extern "C" wp_status wp_static_status(wp_stream stream, double timeout_s)
{
    void *base = nullptr;
    cudaError_t e = static_base(&base);
    if (e != cudaSuccess)
        return static_fail(WP_ERR_CUDA, "looking up the static scratch (cudaGetSymbolAddress) failed", e);
    const wp_status st = wp_stream_status(nullptr, stream, timeout_s);
    if (st != WP_OK) return st;
    int flag = 0;
    e = cudaMemcpy(&flag, base, sizeof flag, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return static_fail(WP_ERR_CUDA, "reading the static error flag failed", e);
    if (flag) return static_fail(WP_ERR_TIMEOUT, "a device wait of wp_probe_accumulate_static gave up");
    return WP_OK;
}
