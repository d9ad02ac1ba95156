// Small element-wise and reduction kernels around the time loop: the per-point factor
// dt^2/m, buffer fills, the sum of per-shot images, model validation and the residual /
// misfit J = 1/2 sum (d_syn - d_obs)^2.
#include <atomic>
#include <utility>
#include <vector>

#include "wp_internal.cuh"

namespace wp {

static std::atomic<long long> g_launches{0};
void count_launch(long long k) { g_launches += k; }
long long launches() { return g_launches.load(); }

// Optional per-kernel-class timing: CUDA events recorded on the launching stream around
// each timed launch, read back after the caller synchronises.
namespace {
struct ProfClass {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    size_t used = 0;
};
bool g_prof = false;
ProfClass g_pc[PROF_NCLASS];
}  // namespace

void prof_enable(int on, int capacity)
{
    g_prof = on != 0;
    for (auto &c : g_pc) {
        c.used = 0;
        while (on && (int)c.ev.size() < capacity) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            c.ev.push_back({a, b});
        }
    }
}

cudaEvent_t prof_begin(int cls, cudaStream_t s)
{
    if (!g_prof || cls < 0 || cls >= PROF_NCLASS) return nullptr;
    ProfClass &c = g_pc[cls];
    if (c.used >= c.ev.size()) return nullptr;
    cudaEventRecord(c.ev[c.used].first, s);
    return c.ev[c.used].first;
}

void prof_end(int cls, cudaEvent_t began, cudaStream_t s)
{
    if (!began) return;
    ProfClass &c = g_pc[cls];
    cudaEventRecord(c.ev[c.used].second, s);
    c.used++;
}

int prof_read(int cls, double *total_ms, long long *count)
{
    if (cls < 0 || cls >= PROF_NCLASS) return -1;
    ProfClass &c = g_pc[cls];
    double t = 0.0;
    for (size_t i = 0; i < c.used; i++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c.ev[i].first, c.ev[i].second) != cudaSuccess) return -1;
        t += ms;
    }
    *total_ms = t;
    *count = (long long)c.used;
    return 0;
}

static unsigned grid_for(long long n, int bs)
{
    long long g = (n + bs - 1) / bs;
    const long long cap = 152LL * 64;  // grid-stride beyond 64 blocks per SM
    return (unsigned)(g < cap ? (g > 0 ? g : 1) : cap);
}

// b = dt^2/m on the padded internal layout (row pitch NXp); pad columns hold 0.
__global__ void b_field_kernel(const float *m, double dt2, long long Np, int NX, int NXp, float *b)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < Np;
         p += (long long)gridDim.x * blockDim.x) {
        const long long row = p / NXp;
        const int x = (int)(p - row * NXp);
        b[p] = x < NX ? (float)(dt2 / (double)m[row * NX + x]) : 0.f;
    }
}

cudaError_t launch_b_field(const float *m, double dt2, const GridDev &G, float *b, cudaStream_t s)
{
    b_field_kernel<<<grid_for(G.Np, 256), 256, 0, s>>>(m, dt2, G.Np, G.NX, G.NXp, b);
    count_launch();
    return cudaGetLastError();
}

__global__ void fill_kernel(float *p, long long n, float v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

cudaError_t launch_fill(float *p, long long n, float v, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, n, v);
    count_launch();
    return cudaGetLastError();
}

// g[p] = sum_s img[s][p'] in shot order (deterministic); p' = p, or p mapped to the
// padded pitch when the images use the internal layout.
__global__ void shot_sum_kernel(const float *img, long long img_ss, int nshots, long long N,
                                int NX, int NXp, int padded, float *g)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        long long q = p;
        if (padded) {
            const long long row = p / NX;
            q = row * NXp + (p - row * NX);
        }
        float acc = 0.f;
        for (int s = 0; s < nshots; s++) acc += img[(long long)s * img_ss + q];
        g[p] = acc;
    }
}

cudaError_t launch_shot_sum(const float *img, long long img_ss, int nshots, const GridDev &G,
                            bool padded, float *g, cudaStream_t s)
{
    shot_sum_kernel<<<grid_for(G.N, 256), 256, 0, s>>>(img, img_ss, nshots, G.N, G.NX, G.NXp,
                                                       padded ? 1 : 0, g);
    count_launch();
    return cudaGetLastError();
}

// out2 = {min m, max m} over finite positive values; *bad counts non-positive/non-finite.
__global__ void minmax_kernel(const float *m, long long N, float *out2, int *bad)
{
    __shared__ float smin[256], smax[256];
    __shared__ int sbad[256];
    float lo = 3.4e38f, hi = 0.f;
    int nb = 0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        const float x = m[p];
        if (!(x > 0.f) || !isfinite(x)) nb++;
        else {
            lo = fminf(lo, x);
            hi = fmaxf(hi, x);
        }
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    sbad[threadIdx.x] = nb;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + w]);
            smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + w]);
            sbad[threadIdx.x] += sbad[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // Positive floats order like their bit patterns, so integer atomics give min/max.
        atomicMin((int *)&out2[0], __float_as_int(smin[0]));
        atomicMax((int *)&out2[1], __float_as_int(smax[0]));
        atomicAdd(bad, sbad[0]);
    }
}

cudaError_t launch_minmax(const float *m, long long N, float *out2, int *bad, cudaStream_t s)
{
    unsigned g = grid_for(N, 256);
    if (g > 1024) g = 1024;
    minmax_kernel<<<g, 256, 0, s>>>(m, N, out2, bad);
    count_launch();
    return cudaGetLastError();
}

// out[0] = max(0, max_i x[i]) (non-negative floats order like their bit patterns).
__global__ void maxval_kernel(const float *x, long long n, float *out)
{
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, x[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax((int *)out, __float_as_int(m));
}

// *count += the number of i with a[i] > b[i] or either value not finite.
__global__ void count_greater_kernel(const float *a, const float *b, long long n, int *count)
{
    int c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        c += !(a[i] <= b[i]) || !isfinite(a[i]) || !isfinite(b[i]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

cudaError_t launch_count_greater(const float *a, const float *b, long long n, int *count, cudaStream_t s)
{
    unsigned g = grid_for(n, 256);
    if (g > 1024) g = 1024;
    count_greater_kernel<<<g, 256, 0, s>>>(a, b, n, count);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_maxval(const float *x, long long n, float *out, cudaStream_t s)
{
    unsigned g = grid_for(n, 256);
    if (g > 1024) g = 1024;
    maxval_kernel<<<g, 256, 0, s>>>(x, n, out);
    count_launch();
    return cudaGetLastError();
}

// One thread waits on an mbarrier that nothing completes; the bounded wait gives up, sets
// the flag and returns (the failure path of every device wait in this library).
__global__ void bounded_wait_kernel(int *err)
{
    __shared__ uint64_t bar;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait_bounded(&bar, 0)) atomicExch(err, 1);
}

cudaError_t launch_bounded_wait(int *err, cudaStream_t s)
{
    bounded_wait_kernel<<<1, 1, 0, s>>>(err);
    count_launch();
    return cudaGetLastError();
}

int residual_parts(long long n)
{
    long long g = (n + 255) / 256;
    return (int)(g < 1024 ? (g > 0 ? g : 1) : 1024);
}

// res = a - b; partials[block] = sum over the block's grid-stride range of res^2 (double).
// vec4: a, b and res (if any) 16-byte aligned: the first n / 4 * 4 entries go as float4, the
// four squares of a float4 summed in FP32 and added to the thread's FP64 sum (one FP64 add
// per four entries), the rest one by one.
template <bool vec4>
__global__ void residual_kernel(const float *a, const float *b, float *res, long long n,
                                double *partials)
{
    __shared__ double sacc[256];
    double acc = 0.0;
    const long long n4 = vec4 ? n / 4 : 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 x = __ldg((const float4 *)a + i), y = __ldg((const float4 *)b + i);
        const float4 r = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
        if (res) ((float4 *)res)[i] = r;
        acc += (double)(r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w);
    }
    for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float r = a[i] - b[i];
        if (res) res[i] = r;
        acc += (double)r * (double)r;
    }
    sacc[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sacc[threadIdx.x] += sacc[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && partials) partials[blockIdx.x] = sacc[0];
}

__global__ void finish_misfit_kernel(const double *partials, int nparts, double *misfit)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double acc = 0.0;
        for (int i = 0; i < nparts; i++) acc += partials[i];
        *misfit = 0.5 * acc;
    }
}

cudaError_t launch_residual(const float *a, const float *b, float *res, long long n,
                            double *partials, int nparts, double *misfit, cudaStream_t s)
{
    const bool v4 = !((uintptr_t)a & 15) && !((uintptr_t)b & 15) && !((uintptr_t)res & 15);
    if (v4) residual_kernel<true><<<nparts, 256, 0, s>>>(a, b, res, n, misfit ? partials : nullptr);
    else residual_kernel<false><<<nparts, 256, 0, s>>>(a, b, res, n, misfit ? partials : nullptr);
    count_launch();
    if (misfit) {
        finish_misfit_kernel<<<1, 32, 0, s>>>(partials, nparts, misfit);
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace wp
