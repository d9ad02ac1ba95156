// Probe accumulation on the tensor cores (Eq. 3): for one block of buffered time steps,
//   P[i][x] += scale * sum_t A[t][x] * Q[t0 + t][i]
// an [N x Tb] . [Tb x r] contraction per shot.  A is read from the time-step ring written
// by the stencil (forward: u_tt rebuilt from two stored increments; adjoint: v itself),
// split into bfloat16 hi + lo in registers and stored in the K-major 128-byte-swizzled
// layout that tcgen05.mma reads; the probes arrive pre-split (hi/lo) in global memory.
// Four bf16 products (hi*hi, lo*hi, hi*lo, lo*lo) accumulate in FP32 in tensor memory,
// which keeps the contraction faithful to FP32 (relative error ~2^-17) for any probe
// matrix, Rademacher or orthonormal.  One CTA owns 128 grid points (M = 128) and all r
// probes (N = r rounded up to 16); K runs over the block in chunks of 64 time steps.
//
// After the last adjoint block the epilogue also forms the randomized imaging condition
// img[x] = img_scale * sum_i Pu[i][x] * Pv[i][x] (Eq. 3) while P_v is still in registers.
#include "wp_internal.cuh"

namespace wp {

constexpr int KCH = 64;  // time steps per K chunk: one 128-byte swizzle row of bf16

__host__ __device__ inline uint32_t tmem_cols_for(int r_pad)
{
    uint32_t c = 32;
    while (c < (uint32_t)r_pad) c <<= 1;
    return c;
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo_k, __nv_bfloat16 hi_k)
{
    return (uint32_t)__bfloat16_as_ushort(lo_k) | ((uint32_t)__bfloat16_as_ushort(hi_k) << 16);
}

__global__ void __launch_bounds__(128) probe_gemm_kernel(const GemmArgs A)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // stays a shared pointer
    uint8_t *a_hi = smem;
    uint8_t *a_lo = smem + 16384;
    uint8_t *b_hi = smem + 32768;
    uint8_t *b_lo = b_hi + A.r_pad * 128;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;

    const int tile = blockIdx.x, shot = blockIdx.y, m = threadIdx.x, warp = m >> 5;
    const long long p = (long long)tile * 128 + m;
    const bool valid = p < A.N;
    const uint32_t ncols = tmem_cols_for(A.r_pad);

    if (warp == 0) tmem_alloc(&tmem_holder, ncols);
    if (m == 0) {
        mbar_init(&mbar, 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;

    float cp = 1.f, cm = 1.f;
    if (A.mode == 1 && valid) {
        const long long PS = (long long)A.G.NX * A.G.NY;
        const int z = (int)(p / PS);
        const long long rem = p - (long long)z * PS;
        const int y = (int)(rem / A.G.NX), x = (int)(rem - (long long)y * A.G.NX);
        const float sd = damp_at(A.G, x, y, z);
        cp = 1.f + sd;
        cm = 1.f - sd;
    }
    const float *ring = A.ring + (long long)shot * A.ring_ss + (valid ? p : 0);
    const __nv_bfloat16 *qh = A.qhi + (long long)shot * A.q_ss;
    const __nv_bfloat16 *ql = A.qlo + (long long)shot * A.q_ss;
    const uint32_t idesc = idesc_bf16_f32(128, A.r_pad);
    const int nchunks = (A.cnt + KCH - 1) / KCH;
    uint32_t phase = 0;

    for (int c = 0; c < nchunks; c++) {
        const int tb = c * KCH;
        float v[KCH];
        int slot = (A.slot0 + tb) % A.nslots;
        if (A.mode == 0) {
#pragma unroll
            for (int t = 0; t < KCH; t++) {
                v[t] = (valid && tb + t < A.cnt) ? ring[(long long)slot * A.N] : 0.f;
                slot = (slot + 1 == A.nslots) ? 0 : slot + 1;
            }
        } else {
            float prev = (valid && tb < A.cnt) ? ring[(long long)slot * A.N] : 0.f;
#pragma unroll
            for (int t = 0; t < KCH; t++) {
                slot = (slot + 1 == A.nslots) ? 0 : slot + 1;
                const bool in = valid && tb + t < A.cnt;
                const float nx = in ? ring[(long long)slot * A.N] : 0.f;
                v[t] = in ? cp * nx - cm * prev : 0.f;
                prev = nx;
            }
        }
#pragma unroll
        for (int cc = 0; cc < 8; cc++) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float x0 = v[cc * 8 + 2 * j], x1 = v[cc * 8 + 2 * j + 1];
                const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
                const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
                const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
                h[j] = pack_bf16(h0, h1);
                l[j] = pack_bf16(l0, l1);
            }
            const uint32_t off = (uint32_t)m * 128u + ((uint32_t)(cc ^ (m & 7)) << 4);
            *(uint4 *)(a_hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
            *(uint4 *)(a_lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
        }
        for (int idx = m; idx < A.r_pad * 8; idx += 128) {
            const int i = idx >> 3, cc = idx & 7;
            const long long g = (long long)i * A.nt_pad + A.t0 + tb + cc * 8;
            const uint4 h = *(const uint4 *)(qh + g);
            const uint4 l = *(const uint4 *)(ql + g);
            const uint32_t off = (uint32_t)i * 128u + ((uint32_t)(cc ^ (i & 7)) << 4);
            *(uint4 *)(b_hi + off) = h;
            *(uint4 *)(b_lo + off) = l;
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (m == 0) {
            tc_fence_after();
            const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo);
            const uint32_t bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
            for (int k = 0; k < KCH / 16; k++) {
                const uint32_t ko = (uint32_t)k * 32u;
                const uint64_t dah = sdesc_k_sw128(ah + ko), dal = sdesc_k_sw128(al + ko);
                const uint64_t dbh = sdesc_k_sw128(bh + ko), dbl = sdesc_k_sw128(bl + ko);
                umma_bf16(tmem, dah, dbh, idesc, (c > 0 || k > 0) ? 1u : 0u);
                umma_bf16(tmem, dal, dbh, idesc, 1u);
                umma_bf16(tmem, dah, dbl, idesc, 1u);
                umma_bf16(tmem, dal, dbl, idesc, 1u);
            }
            umma_commit(&mbar);
        }
        if (!mbar_wait_bounded(&mbar, phase)) abort_flag = 1;
        phase ^= 1;
        __syncthreads();
        if (abort_flag) break;
    }

    if (!abort_flag) {
        tc_fence_after();
        float *P = A.P + (long long)shot * A.P_ss;
        const float *Pu = A.do_img ? A.Pu + (long long)shot * A.Pu_ss : nullptr;
        float img = 0.f;
        for (int c0 = 0; c0 < A.r_pad; c0 += 16) {
            uint32_t r16[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r16);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int i = c0 + j;
                if (i < A.r && valid) {
                    float *dst = P + (long long)i * A.N + p;
                    const float nv = *dst + A.scale * __uint_as_float(r16[j]);
                    *dst = nv;
                    if (Pu) img += Pu[(long long)i * A.N + p] * nv;
                }
            }
        }
        if (Pu && valid) A.img[(long long)shot * A.img_ss + p] = A.img_scale * img;
    } else {
        if (m == 0) atomicExch(A.err, 1);
        // Give in-flight MMAs one more bounded chance to retire, then free the TMEM whether
        // or not they did: a block that exits still holding its columns leaves them
        // allocated for the rest of the context, so every later launch that allocates on
        // this SM would wait forever.  The cost of freeing is that an MMA still in flight
        // could write columns a block of a later launch has just allocated; the error flag
        // this call reports tells the caller that results computed on the stream since then
        // are suspect.
        mbar_wait_bounded(&mbar, phase ^ 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

size_t probe_gemm_smem(int r_pad)
{
    const size_t need = 1024 + 32768 + (size_t)2 * r_pad * 128;
    // Keep (co-resident CTAs) x (TMEM columns) within the 512 columns of an SM.
    const int max_ctas = 512 / (int)tmem_cols_for(r_pad);
    const size_t cap = (size_t)233472 / (size_t)(max_ctas + 1) + 1024;
    return need > cap ? need : cap;
}

cudaError_t launch_probe_gemm(const GemmArgs &A, int nshots, cudaStream_t s)
{
    const size_t smem = probe_gemm_smem(A.r_pad);
    cudaError_t e = cudaFuncSetAttribute(probe_gemm_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((A.N + 127) / 128), nshots);
    cudaEvent_t ev = prof_begin(PROF_GEMM, s);
    probe_gemm_kernel<<<grid, 128, smem, s>>>(A);
    prof_end(PROF_GEMM, ev, s);
    count_launch();
    return cudaGetLastError();
}

// Q [shot][nt][r] (fp32)  ->  qhi/qlo [shot][r_pad][nt_pad] (bf16, zero padded).
__global__ void probe_split_kernel(const float *Q, int nt, int r, int r_pad, int nt_pad,
                                   __nv_bfloat16 *qhi, __nv_bfloat16 *qlo)
{
    const int shot = blockIdx.z, i = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt_pad) return;
    float x = 0.f;
    if (i < r && t < nt) x = Q[((long long)shot * nt + t) * r + i];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    const long long o = ((long long)shot * r_pad + i) * nt_pad + t;
    qhi[o] = h;
    qlo[o] = l;
}

cudaError_t launch_probe_split(const float *Q, int nshots, int nt, int r, int r_pad, int nt_pad,
                               __nv_bfloat16 *qhi, __nv_bfloat16 *qlo, cudaStream_t s)
{
    dim3 grid((nt_pad + 255) / 256, r_pad, nshots);
    probe_split_kernel<<<grid, 256, 0, s>>>(Q, nt, r, r_pad, nt_pad, qhi, qlo);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
