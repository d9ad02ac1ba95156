// Subsurface-offset image volume from the probed projections (Eq. 4):
//   out[h + nh][p] = scale * sum_s sum_i P_u[s][i][p + h] * P_v[s][i][p - h],  h = -nh .. nh,
// with the offset along x (the fastest axis) and zero wherever p + h or p - h leaves the
// row.  Offset 0 is the randomized image of Eq. 3.
//
// A block owns 128 consecutive x of one (z, y) row and all offsets: thread (xg, hg) keeps
// XT = 4 consecutive x-positions and HT = 16 consecutive offsets (64 sums) in registers.
// Probe rows of P_u and P_v are staged through shared memory 16 probes at a time in two
// buffers (4-byte cp.async, zero-filled outside the row), the next chunk in flight while
// the current one is used.  For one probe a thread reads the 19 values of P_u and of P_v
// its 64 products need with five 16-byte shared loads each (the staging offsets of the two
// rows are chosen so that both windows start on a 16-byte boundary): 64 FMAs per 10 loads.
// (8 x-positions per thread give 128 FMAs per 12 loads but 192 registers; measured slower.)
#include "wp_internal.cuh"

namespace wp {

namespace {
constexpr int OX = 128;   // x positions per block
#ifndef WP_OFF_XT
#define WP_OFF_XT 4
#endif
#ifndef WP_OFF_PC
#define WP_OFF_PC 16
#endif
constexpr int XT = WP_OFF_XT;   // x positions per thread (4 or 8)
constexpr int HT = 16;          // offsets per thread
constexpr int PC = WP_OFF_PC;   // probes per shared-memory chunk

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool ok)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 4 : 0)
                 : "memory");
}

// offset groups of HT, padded to an even count (two groups per warp)
__host__ __device__ inline int offset_groups(int nh) { return ((2 * nh + 1 + HT - 1) / HT + 1) / 2 * 2; }
__host__ __device__ inline int window_len(int nh) { return HT * offset_groups(nh) + OX; }
}  // namespace

__global__ void __launch_bounds__(OX / XT * 10) offset_image_kernel(const float *__restrict__ Pu, const float *__restrict__ Pv,
                                                                    int NX, long long N, int ntx, int r, int nshots,
                                                                    float scale, int nh, float *__restrict__ out)
{
    extern __shared__ float4 sm4[];
    float *sm = (float *)sm4;
    const int NG = offset_groups(nh);
    const int L = window_len(nh);                 // staged row length (a multiple of 4)
    // row j of the P_u buffer holds x0 - OFU + j, of the P_v buffer x0 - OFV + j
    const int OFU = nh, OFV = HT * NG - nh - 1;
    float *su = sm, *sv = sm + PC * L;
    const int tid = threadIdx.x, xg = tid & (OX / XT - 1), hg = tid / (OX / XT);
    const long long row = blockIdx.x / ntx;
    const int x0 = (int)(blockIdx.x % ntx) * OX;
    const long long rb = row * NX;
    const int xt = XT * xg;
    const int h0 = -nh + hg * HT;
    float acc[XT][HT];
#pragma unroll
    for (int a = 0; a < XT; a++)
#pragma unroll
        for (int b = 0; b < HT; b++) acc[a][b] = 0.f;

    const int nrc = (r + PC - 1) / PC;   // probe chunks per shot
    const int nchunks = nshots * nrc;
    auto issue = [&](int c) {
        const int s = c / nrc, i0 = (c - s * nrc) * PC;
        float *bu = su + (c & 1) * (2 * PC * L), *bv = bu + PC * L;
#pragma unroll
        for (int pi = 0; pi < PC; pi++) {
            const bool iok = i0 + pi < r;
            const long long base = ((long long)s * r + min(i0 + pi, r - 1)) * N + rb;
            for (int j = tid; j < L; j += blockDim.x) {
                const int xu = x0 - OFU + j, xv = x0 - OFV + j;
                const bool oku = iok && xu >= 0 && xu < NX, okv = iok && xv >= 0 && xv < NX;
                // a valid address even where nothing is copied
                cp_async4(bu + pi * L + j, Pu + base + min(max(xu, 0), NX - 1), oku);
                cp_async4(bv + pi * L + j, Pv + base + min(max(xv, 0), NX - 1), okv);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    issue(0);
    for (int c = 0; c < nchunks; c++) {
        if (c + 1 < nchunks) issue(c + 1);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // chunk c has landed (own copies)
        __syncthreads();                                       // ... and everyone's
        const int s = c / nrc, i0 = (c - s * nrc) * PC;
        const float *bu = su + (c & 1) * (2 * PC * L), *bv = bu + PC * L;
        const int np = min(PC, r - i0);
        for (int pi = 0; pi < np; pi++) {
            // U[k] = P_u at x0 + xt + h0 + k; V[k] = P_v at x0 + xt - h0 - (HT - 1) + k
            const float4 *u4 = (const float4 *)(bu + pi * L + OFU + xt + h0);
            const float4 *v4 = (const float4 *)(bv + pi * L + OFV + xt - h0 - (HT - 1));
            float U[XT + HT], V[XT + HT];
#pragma unroll
            for (int q = 0; q < (XT + HT) / 4; q++) {
                const float4 a = u4[q], b = v4[q];
                U[4 * q] = a.x; U[4 * q + 1] = a.y; U[4 * q + 2] = a.z; U[4 * q + 3] = a.w;
                V[4 * q] = b.x; V[4 * q + 1] = b.y; V[4 * q + 2] = b.z; V[4 * q + 3] = b.w;
            }
            // the pair of offset h0 + hh at x0 + xt + xx: P_u[x + h] * P_v[x - h]
#pragma unroll
            for (int xx = 0; xx < XT; xx++)
#pragma unroll
                for (int hh = 0; hh < HT; hh++) acc[xx][hh] = fmaf(U[xx + hh], V[xx - hh + HT - 1], acc[xx][hh]);
        }
        __syncthreads();   // buffer c & 1 is refilled by the issue of chunk c + 2
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
    for (int hh = 0; hh < HT; hh++) {
        const int h = h0 + hh;
        if (h > nh) break;
#pragma unroll
        for (int xx = 0; xx < XT; xx++) {
            const int x = x0 + xt + xx;
            if (x < NX) out[(long long)(h + nh) * N + rb + x] = scale * acc[xx][hh];
        }
    }
}

cudaError_t launch_offset_image(const float *Pu, const float *Pv, int NX, long long N, int r,
                                int nshots, float scale, int nh, float *out, cudaStream_t s)
{
    const long long rows = N / NX;
    const int ntx = (NX + OX - 1) / OX;
    const long long blocks = rows * ntx;
    if (blocks >= (1LL << 31)) return cudaErrorInvalidValue;
    const int threads = OX / XT * offset_groups(nh);
    const size_t smem = (size_t)4 * PC * window_len(nh) * sizeof(float);   // 2 buffers x (u, v)
    cudaFuncSetAttribute(offset_image_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    offset_image_kernel<<<(unsigned)blocks, threads, smem, s>>>(Pu, Pv, NX, N, ntx, r, nshots, scale, nh, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
