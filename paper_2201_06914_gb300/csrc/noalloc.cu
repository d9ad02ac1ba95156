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
#include <mutex>

#include "wp_internal.cuh"

namespace {

// Fixed scratch: 16 MiB on every device that loads libwp.so.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device ordinal.  In host code the array's name
// is only a host-side stand-in, so the real address is looked up once per device with
// cudaGetSymbolAddress while that device is current.
constexpr int kMaxDevices = 64;
void *g_static_ptr[kMaxDevices] = {};
std::mutex g_static_mtx;

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
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(WP_ERR_CUDA, "cudaGetDevice failed", e);
    if (dev < 0 || dev >= kMaxDevices) return static_fail(WP_ERR_INVALID, "device ordinal too large");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mtx);
        if (!g_static_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p)
                return static_fail(WP_ERR_CUDA, "cudaGetSymbolAddress(g_static_scratch) failed", e);
            g_static_ptr[dev] = p;
        }
        base = g_static_ptr[dev];
    }
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
