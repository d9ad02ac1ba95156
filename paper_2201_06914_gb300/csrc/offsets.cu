// Subsurface-offset image volume from the probed projections (Eq. 4):
//   out[h + nh][p] = scale * sum_s sum_i P_u[s][i][p + h] * P_v[s][i][p - h],  h = -nh .. nh,
// with the offset along x (the fastest axis) and zero wherever p + h or p - h leaves the
// row.  Offset 0 is the randomized image of Eq. 3.
//
// A block owns 128 consecutive x of one (z, y) row and all offsets: thread (xg, hg) keeps
// the 4 x-positions 4*xg .. 4*xg+3 and HT consecutive offsets in registers.  Probe rows of
// P_u and P_v are staged through shared memory 8 probes at a time in two buffers (4-byte
// cp.async, zero-filled outside the row), the next chunk in flight while the current one is
// used; windows extend nh + HT points on both sides.  Along the offsets the thread slides two
// 4-wide register windows in opposite directions (u[x + h] moves right, v[x - h] moves
// left), so each step costs 2 shared loads for 4 FMAs.
#include "wp_internal.cuh"

namespace wp {

namespace {
constexpr int OX = 128;   // x positions per block
constexpr int HT = 21;    // offsets per thread
constexpr int PC = 8;     // probes per shared-memory chunk

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool ok)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 4 : 0)
                 : "memory");
}
}  // namespace

__global__ void offset_image_kernel(const float *__restrict__ Pu, const float *__restrict__ Pv, int NX,
                                    long long N, int ntx, int r, int nshots, float scale, int nh,
                                    float *__restrict__ out)
{
    extern __shared__ float sm[];
    const int OFF = nh + HT;                      // window starts at x0 - OFF
    const int L = OX + 2 * OFF + 4;               // window length
    float *su = sm, *sv = sm + PC * L;
    const int tid = threadIdx.x, xg = tid & 31, hg = tid >> 5;
    const long long row = blockIdx.x / ntx;
    const int x0 = (int)(blockIdx.x % ntx) * OX;
    const long long rb = row * NX;
    const int xt = 4 * xg;
    const int h0 = -nh + hg * HT;
    float acc[4][HT];
#pragma unroll
    for (int a = 0; a < 4; a++)
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
                const int x = x0 - OFF + j;
                const bool ok = iok && x >= 0 && x < NX;
                const int xc = min(max(x, 0), NX - 1);   // a valid address even where nothing is copied
                cp_async4(bu + pi * L + j, Pu + base + xc, ok);
                cp_async4(bv + pi * L + j, Pv + base + xc, ok);
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
            const float *u = bu + pi * L + OFF + xt + h0;   // u[k] = P_u at x0 + xt + h0 + k
            const float *v = bv + pi * L + OFF + xt - h0;   // v[k] = P_v at x0 + xt - h0 + k
            float uw[4], vw[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                uw[q] = u[q];
                vw[q] = v[q];
            }
#pragma unroll
            for (int hh = 0; hh < HT; hh++) {
                // uw[xx] = u[xx + hh], vw[xx] = v[xx - hh]: the pair of offset h0 + hh at x + xx
#pragma unroll
                for (int xx = 0; xx < 4; xx++) acc[xx][hh] = fmaf(uw[xx], vw[xx], acc[xx][hh]);
                if (hh + 1 < HT) {
                    uw[0] = uw[1];
                    uw[1] = uw[2];
                    uw[2] = uw[3];
                    uw[3] = u[hh + 4];
                    vw[3] = vw[2];
                    vw[2] = vw[1];
                    vw[1] = vw[0];
                    vw[0] = v[-hh - 1];
                }
            }
        }
        __syncthreads();   // buffer c & 1 is refilled by the issue of chunk c + 2
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
#pragma unroll
    for (int hh = 0; hh < HT; hh++) {
        const int h = h0 + hh;
        if (h > nh) break;
#pragma unroll
        for (int xx = 0; xx < 4; xx++) {
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
    const int hgroups = (2 * nh + 1 + HT - 1) / HT;
    const size_t smem = (size_t)4 * PC * (OX + 2 * (nh + HT) + 4) * sizeof(float);   // 2 buffers x (u, v)
    offset_image_kernel<<<(unsigned)blocks, 32 * hgroups, smem, s>>>(Pu, Pv, NX, N, ntx, r, nshots, scale,
                                                                    nh, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
