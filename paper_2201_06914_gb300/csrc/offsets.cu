// Subsurface-offset image volume from the probed projections (Eq. 4) on the tensor cores:
//   out[h + nh][p] = scale * sum_s sum_i P_u[s][i][p + h] * P_v[s][i][p - h],  h = -nh .. nh,
// with the offset along x (the fastest axis) and zero wherever p + h or p - h leaves the
// row.  Offset 0 is the randomized image of Eq. 3.
//
// Per (z, y) row the volume is a band of the Gram matrix G = P_u^T P_v of the row, the
// contraction running over k = (shot, probe): out[h][p] = G[p + h][p - h], the entries with
// a - b = 2h, |a - b| <= 2 nh.  A work item owns 128 consecutive a (= p + h) of one row and
// the NB = 128 + 4 nh (rounded up to 16) columns b in [a0 - 2 nh, a0 + 128 + 2 nh), and
// computes that 128 x NB block of G as one tcgen05 accumulator in tensor memory:
//   warps 0-7   converters: per 64-k chunk, bring the block's P_u rows (128 a) and P_v
//               rows (NB b) from global memory (coalesced along x), split FP32 into bf16
//               hi + lo and store them in the K-major 128-byte-swizzled layout of tcgen05.
//               Dense operands (rows N floats apart, no alignment): 4-byte loads into
//               registers, two blocks of 32 in flight per thread.  Row-aligned operands
//               (rows 512-byte aligned, points at a pitch of 4): the chunk arrives by TMA
//               (three tiled copies) in an FP32 staging area while the previous chunk's
//               MMAs run, and the converters read it from shared memory;
//   warps 8-11  epilogue: tcgen05.ld of the accumulator in 16-column slices; each lane (one
//               a) keeps the columns of its band with a - b even and writes
//               out[h][a - h] = scale * G[a][b], h = (a - b) / 2.  Before its share of an
//               item's epilogue, lane 0 of warp 8 issues the item's MMAs: 4 products
//               (hi*hi, lo*hi, hi*lo, lo*lo) per 16-k slice for each of the at most two
//               N <= 256 halves, FP32 accumulation.  The accumulator is single-buffered
//               (128 x NB FP32 columns), so an item's MMAs wait for the previous item's
//               epilogue anyway; taking the issue into an epilogue warp keeps the block at
//               12 warps (3 per SM sub-partition), which leaves the converters 168
//               registers a thread to keep two blocks of loads in flight.
// Every output (p, h) comes from exactly one a = p + h, so items write disjoint entries;
// the entries with p + h outside [0, NX) belong to no item and stay at the zero the
// launcher writes first.  The bf16 hi/lo split carries 16 significant bits of each
// operand: relative error about 3.5e-6 on random projections (FP32 emulation on the CPU).
// Waits are bounded; a wait that gives up raises the error flag and every role leaves.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "wp_internal.cuh"

namespace wp {

namespace {

constexpr int OT_THREADS = 384;           // warps 0-7 converters, 8-11 epilogue (+ MMA issue)
constexpr int OCONV = 256;
constexpr int OW_EPI = 8;
constexpr int KC = 64;                    // k per chunk: one 128-byte row of bf16
constexpr uint32_t A_BYTES = 128u * 128u; // one bf16 operand of 128 rows x 64 k

struct OffArgs {
    const float *Pu, *Pv;
    int NX, XP;             // points per x-row; x pitch of the operands (NX dense, NXp aligned)
    long long N;            // points of the model (out holds 2 nh + 1 rows of N)
    long long pitch;        // floats between the probe rows of the operands
    long long rows;         // (z, y) rows
    int ntx;                // 128-point tiles per row
    int K;                  // nshots * r
    int nh, boff;           // offsets per side; a0 - b0 (2 nh, rounded up to 4 when aligned)
    int NB, N1;             // accumulator columns, first MMA half
    float scale;
    float *out;
    int *err;
};

__host__ __device__ inline int off_boff(int nh, bool aligned) { return aligned ? (2 * nh + 3) & ~3 : 2 * nh; }
__host__ __device__ inline int off_nb(int nh, int boff) { return (128 + boff + 2 * nh + 15) / 16 * 16; }
__host__ __device__ inline uint32_t off_stage_bytes(int NB) { return 2u * A_BYTES + 2u * (uint32_t)NB * 128u; }

// Row-aligned operands as 2-D tensors [k][point] (rows `pitch` floats apart): P_u in boxes
// of 128 points x 64 k, P_v in two boxes of NB / 2 points x 64 k per chunk.
struct OffMaps {
    CUtensorMap pu, pv;
};

__device__ __forceinline__ void off_tma_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace

template <bool AL>
__global__ void __launch_bounds__(OT_THREADS, 1)
    offset_tc_kernel(const OffArgs A, int ST, const __grid_constant__ OffMaps TM)
{
    extern __shared__ uint8_t smem_raw[];
    // aligned by pointer arithmetic on the shared array (no integer round trip), so the
    // compiler keeps every access derived from it in the shared state space
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ uint64_t full[4], empty[4], accfull, accempty, fbar;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t SB = off_stage_bytes(A.NB);
    const uint32_t ncols = A.NB > 256 ? 512 : 256;
    const long long nitems = A.rows * A.ntx;
    const int nch = (A.K + KC - 1) / KC;

    if (tid == 0) {
        for (int s = 0; s < ST; s++) {
            mbar_init(&full[s], OCONV);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accfull, 1);
        mbar_init(&accempty, 128);
        mbar_init(&fbar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == OW_EPI) tmem_alloc(&tmem_holder, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    auto stage_ptr = [&](int s) { return smem + (size_t)s * SB; };

    if (warp < OW_EPI) {
      if constexpr (AL) {
        // ---------------- converters, row-aligned operands ----------------
        // The chunk's FP32 rows arrive by TMA in a staging area after the operand stage
        // (one stage, ST == 1): P_u as [64 k][128 points], P_v as two [64 k][NB / 2 points]
        // tiles.  Thread (m, half) converts operand row m of each 128-row block for k in its
        // half: 32 shared loads along k (a warp reads 32 consecutive points per load), the
        // hi/lo split, and the swizzled K-major stores of the dense path.  Points outside
        // the x-row (the tiles run into the neighbouring rows) are zeroed here.  Once every
        // converter has read the staging area, thread 0 starts the next chunk's copies,
        // which land while the MMA of this chunk runs.
        const int m = tid & 127, half = tid >> 7;
        const int nbb = (A.NB + 127) / 128;
        const int NBh = A.NB / 2;
        const float *F = (const float *)stage_ptr(ST);
        const uint32_t fbytes = (128u + (uint32_t)A.NB) * KC * 4u;
        const long long myitems = ((long long)nitems - blockIdx.x + gridDim.x - 1) / gridDim.x;
        const long long total = myitems * nch;   // chunks of this CTA
        auto issue = [&](long long j) {
            const long long item = blockIdx.x + (j / nch) * (long long)gridDim.x;
            const int c = (int)(j % nch);
            const long long row = item / A.ntx;
            const int a0 = (int)(item - row * A.ntx) * 128;
            const int xa = (int)(row * A.XP) + a0, xb = xa - A.boff;
            uint8_t *f = stage_ptr(ST);
            mbar_arrive_expect_tx(&fbar, fbytes);
            off_tma_2d(f, &TM.pu, xa, c * KC, &fbar);
            off_tma_2d(f + 128 * KC * 4, &TM.pv, xb, c * KC, &fbar);
            off_tma_2d(f + (size_t)(128 + NBh) * KC * 4, &TM.pv, xb + NBh, c * KC, &fbar);
        };
        auto store = [&](int j, int row_l, const float (&v)[KC / 2]) {
            uint8_t *st = stage_ptr(0);
            uint8_t *hi = j == 0 ? st : st + 2 * A_BYTES;
            uint8_t *lo = j == 0 ? st + A_BYTES : st + 2 * A_BYTES + (size_t)A.NB * 128;
#pragma unroll
            for (int c4 = 0; c4 < 4; c4++) {
                const int cc = half * 4 + c4;   // 16-byte chunk = 8 k of the row
                const uint32_t off = (uint32_t)row_l * 128u + ((uint32_t)(cc ^ (row_l & 7)) << 4);
                const float *xv = v + c4 * 8;
                uint4 h, l;
                split_bf16x2(xv[0], xv[1], h.x, l.x);
                split_bf16x2(xv[2], xv[3], h.y, l.y);
                split_bf16x2(xv[4], xv[5], h.z, l.z);
                split_bf16x2(xv[6], xv[7], h.w, l.w);
                *(uint4 *)(hi + off) = h;
                *(uint4 *)(lo + off) = l;
            }
        };
        long long issued = -1, landed = -1;   // last chunk whose copies were issued / waited for
        if (tid == 0 && total > 0) {
            issue(0);
            issued = 0;
        }
        for (long long j = 0; j < total; j++) {
            const long long item = blockIdx.x + (j / nch) * (long long)gridDim.x;
            const long long row = item / A.ntx;
            const int a0 = (int)(item - row * A.ntx) * 128, b0 = a0 - A.boff;
            // the operand stage is free once the MMA of chunk j - 1 is done; the staging
            // area holds chunk j once its copies have landed
            bool got = mbar_wait_abortable(&empty[0], (uint32_t)(j & 1) ^ 1u, &abort_flag);
            got = got && mbar_wait_abortable(&fbar, (uint32_t)(j & 1), &abort_flag);
            if (got) landed = j;
            if (bar_any<1, OCONV>(!got)) break;
#pragma unroll 1
            for (int jb = 0; jb <= nbb; jb++) {
                const int row_l = jb == 0 ? m : 128 * (jb - 1) + m;
                if (jb > 0 && row_l >= A.NB) break;
                const int x = jb == 0 ? a0 + m : b0 + row_l;
                const bool xin = x >= 0 && x < A.NX;
                const float *src;
                int ld;
                if (jb == 0) {
                    src = F + m;
                    ld = 128;
                } else {
                    const int tl = row_l >= NBh ? 1 : 0;
                    src = F + 128 * KC + tl * NBh * KC + (row_l - tl * NBh);
                    ld = NBh;
                }
                src += (half * (KC / 2)) * ld;
                float v[KC / 2];
#pragma unroll
                for (int t = 0; t < KC / 2; t++) v[t] = xin ? src[t * ld] : 0.f;
                store(jb, row_l, v);
            }
            asm volatile("bar.sync 3, %0;" ::"n"(OCONV) : "memory");   // the staging area is read
            fence_proxy_async_smem();
            mbar_arrive(&full[0]);
            if (tid == 0 && j + 1 < total) {
                issue(j + 1);
                issued = j + 1;
            }
        }
        // after an abort: let copies still in flight land before the block exits
        if (tid == 0 && issued > landed) mbar_wait_bounded(&fbar, (uint32_t)(issued & 1));
      } else {
        // ---------------- converters, dense operands ----------------
        const int m = tid & 127, half = tid >> 7;   // row within a 128-row block, k half
        const int nbb = (A.NB + 127) / 128;         // 128-row blocks of the B operand
        const long long Nr = A.pitch;               // kept in registers
        const int Kr = A.K;
        uint32_t g = 0;
        bool ok = true;
        for (long long item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const long long row = item / A.ntx;
            const int a0 = (int)(item - row * A.ntx) * 128, b0 = a0 - A.boff;
            const long long rb = row * A.XP;
            for (int c = 0; c < nch; c++, g++) {
                const int s = g % ST;
                const bool got = mbar_wait_abortable(&empty[s], ((g / ST) & 1) ^ 1, &abort_flag);
                if (bar_any<1, OCONV>(!got)) {
                    ok = false;
                    break;
                }
                uint8_t *st = stage_ptr(s);
                const int k0 = c * KC + half * (KC / 2);
                // block 0: A rows (P_u at x = a0 + m); blocks 1..: B rows (P_v at b0 + 128 (j-1)
                // + m).  The loads of block j + 1 are issued before block j is converted, so
                // two blocks of 32 loads are in flight per thread (the converters are bound
                // by load latency).
                auto src_of = [&](int j, int &row_l, bool &use, bool &xin) -> const float * {
                    const int x = j == 0 ? a0 + m : b0 + 128 * (j - 1) + m;
                    row_l = j == 0 ? m : 128 * (j - 1) + m;
                    use = j <= nbb && (j == 0 || row_l < A.NB);
                    xin = use && x >= 0 && x < A.NX;
                    return (j == 0 ? A.Pu : A.Pv) + rb + (xin ? x : 0);
                };
                // rows k0 .. k0+31 of one column: a pointer stepped by N (no per-load index
                // multiply), the bound on k checked once for the common full slice
                auto load = [&](const float *src, bool xin, float (&v)[KC / 2]) {
                    const float *q = src + (long long)k0 * Nr;
                    if (xin && k0 + KC / 2 <= Kr) {
#pragma unroll
                        for (int t = 0; t < KC / 2; t++) {
                            v[t] = __ldg(q);
                            q += Nr;
                        }
                    } else {
#pragma unroll
                        for (int t = 0; t < KC / 2; t++) {
                            v[t] = (xin && k0 + t < Kr) ? __ldg(q) : 0.f;
                            if (k0 + t + 1 < Kr) q += Nr;
                        }
                    }
                };
                auto store = [&](int j, int row_l, const float (&v)[KC / 2]) {
                    uint8_t *hi = j == 0 ? st : st + 2 * A_BYTES;
                    uint8_t *lo = j == 0 ? st + A_BYTES : st + 2 * A_BYTES + (size_t)A.NB * 128;
#pragma unroll
                    for (int c4 = 0; c4 < 4; c4++) {
                        const int cc = half * 4 + c4;   // 16-byte chunk = 8 k of the row
                        const uint32_t off = (uint32_t)row_l * 128u + ((uint32_t)(cc ^ (row_l & 7)) << 4);
                        const float *xv = v + c4 * 8;
                        uint4 h, l;
                        split_bf16x2(xv[0], xv[1], h.x, l.x);
                        split_bf16x2(xv[2], xv[3], h.y, l.y);
                        split_bf16x2(xv[4], xv[5], h.z, l.z);
                        split_bf16x2(xv[6], xv[7], h.w, l.w);
                        *(uint4 *)(hi + off) = h;
                        *(uint4 *)(lo + off) = l;
                    }
                };
                float va[KC / 2], vb[KC / 2];
                int ra, rbk;
                bool ua, ub, xa, xb;
                const float *sa = src_of(0, ra, ua, xa);
                load(sa, xa, va);
                for (int j = 0; j <= nbb; j += 2) {
                    const float *sb = src_of(j + 1, rbk, ub, xb);
                    if (ub) load(sb, xb, vb);
                    store(j, ra, va);                       // block j (always used: A or a B block)
                    if (j + 2 <= nbb) {
                        sa = src_of(j + 2, ra, ua, xa);
                        if (ua) load(sa, xa, va);
                        else ua = false;
                    } else {
                        ua = false;
                    }
                    if (ub) store(j + 1, rbk, vb);
                    if (!ua) break;
                }
                fence_proxy_async_smem();
                mbar_arrive(&full[s]);
            }
        }
      }
    } else {
        // ---------------- epilogue (warps 8-11), MMA issue in lane 0 of warp 8 ----------------
        const int ew = warp - OW_EPI;
        const int N2 = A.NB - A.N1;
        const uint32_t id1 = idesc_bf16_f32(128, A.N1), id2 = N2 > 0 ? idesc_bf16_f32(128, N2) : 0u;
        uint32_t gm = 0;   // chunks consumed by the MMA issue
        const int al = ew * 32 + lane;              // a - a0 of this lane
        // columns b - b0 of the warp's band: a - b in [-2 nh, 2 nh], a - b = al + boff - col
        const int c_lo = std::max(0, ew * 32 + A.boff - 2 * A.nh) & ~15;
        const int c_hi = std::min(A.NB, ew * 32 + 32 + A.boff + 2 * A.nh);
        uint32_t j = 0;
        for (long long item = blockIdx.x; item < nitems; item += gridDim.x, j++) {
            const long long row = item / A.ntx;
            const int a0 = (int)(item - row * A.ntx) * 128;
            if (ew == 0) {
                if (lane == 0 && mbar_wait_abortable(&accempty, (j & 1) ^ 1, &abort_flag)) {
                    tc_fence_after();
                    for (int c = 0; c < nch; c++, gm++) {
                        const int s = gm % ST;
                        if (!mbar_wait_abortable(&full[s], (gm / ST) & 1, &abort_flag)) break;
                        tc_fence_after();
                        const uint32_t base = smem_u32(stage_ptr(s));
                        const uint32_t ah = base, al = base + A_BYTES;
                        const uint32_t bh = base + 2 * A_BYTES, bl = bh + (uint32_t)A.NB * 128u;
#pragma unroll
                        for (int k = 0; k < KC / 16; k++) {
                            const uint32_t ko = (uint32_t)k * 32u;
                            const uint64_t dah = sdesc_k_sw128(ah + ko), dal = sdesc_k_sw128(al + ko);
                            const uint32_t acc0 = (c > 0 || k > 0) ? 1u : 0u;
                            {
                                const uint64_t dbh = sdesc_k_sw128(bh + ko), dbl = sdesc_k_sw128(bl + ko);
                                umma_bf16(tmem, dah, dbh, id1, acc0);
                                umma_bf16(tmem, dal, dbh, id1, 1u);
                                umma_bf16(tmem, dah, dbl, id1, 1u);
                                umma_bf16(tmem, dal, dbl, id1, 1u);
                            }
                            if (N2 > 0) {
                                const uint32_t o2 = (uint32_t)A.N1 * 128u;
                                const uint64_t dbh = sdesc_k_sw128(bh + o2 + ko), dbl = sdesc_k_sw128(bl + o2 + ko);
                                const uint32_t t2 = tmem + (uint32_t)A.N1;
                                umma_bf16(t2, dah, dbh, id2, acc0);
                                umma_bf16(t2, dal, dbh, id2, 1u);
                                umma_bf16(t2, dah, dbl, id2, 1u);
                                umma_bf16(t2, dal, dbl, id2, 1u);
                            }
                        }
                        umma_commit(&empty[s]);
                    }
                    if (!abort_flag) umma_commit(&accfull);
                }
                __syncwarp();
            }
            const bool ok = mbar_wait_abortable(&accfull, j & 1, &abort_flag);
            if (bar_any<2, 128>(!ok)) break;
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(ew * 32) << 16);
            float *orow = A.out + row * A.NX;
            for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
                uint32_t r16[16];
                tmem_ld16(taddr + (uint32_t)c0, r16);
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    // column b - b0 = c0 + q; a - b = boff + al - (c0 + q)
                    const int d = al + A.boff - (c0 + q);
                    if (d < -2 * A.nh || d > 2 * A.nh || (d & 1)) continue;
                    const int h = d / 2;
                    const int p = a0 + al - h;
                    if (p < 0 || p >= A.NX) continue;
                    orow[(long long)(h + A.nh) * A.N + p] = A.scale * __uint_as_float(r16[q]);
                }
            }
            tc_fence_before();
            mbar_arrive(&accempty);
        }
    }

    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(A.err, 4);
    if (warp == OW_EPI) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

// Error flag of the offset-volume launches (no workspace is passed to wp_offset_image):
// one int of static device memory per device, cleared by every launch and read by
// offset_status().
__device__ int g_offset_err;

cudaError_t offset_err_ptr(int **p)
{
    return cudaGetSymbolAddress((void **)p, g_offset_err);
}

cudaError_t launch_offset_image(const float *Pu, const float *Pv, bool aligned, int NX, int NXp, long long N,
                                long long pitch, int r, int nshots, float scale, int nh, float *out,
                                cudaStream_t s)
{
    int *err = nullptr;
    cudaError_t e0 = offset_err_ptr(&err);
    if (e0 != cudaSuccess) return e0;
    e0 = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e0 != cudaSuccess) return e0;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    OffArgs A;
    A.Pu = Pu;
    A.Pv = Pv;
    A.NX = NX;
    A.XP = aligned ? NXp : NX;
    A.N = N;
    A.pitch = pitch;
    A.rows = N / NX;
    A.ntx = (NX + 127) / 128;
    A.K = r * nshots;
    A.nh = nh;
    A.boff = off_boff(nh, aligned);
    A.NB = off_nb(nh, A.boff);
    A.N1 = std::min(256, A.NB);
    A.scale = scale;
    A.out = out;
    A.err = err;
    if (A.NB > 512 || (long long)A.K * pitch >= (1LL << 62)) return cudaErrorInvalidValue;
    if (aligned && ((NXp & 3) || (pitch & 3) || ((uintptr_t)Pu & 15) || ((uintptr_t)Pv & 15) ||
                    pitch < A.rows * NXp))
        return cudaErrorInvalidValue;
    const uint32_t SB = off_stage_bytes(A.NB);
    const size_t avail = 227 * 1024 - 1024;
    // aligned: one operand stage plus the FP32 staging area of the same size, when both fit
    // (nh <= 48); wider bands read the aligned rows with the dense path's register loads
    const bool tma = aligned && 2 * (size_t)SB <= avail;
    const int ST = tma ? 1 : (int)std::min<size_t>(4, avail / SB);
    if (ST < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(ST + (tma ? 1 : 0)) * SB + 1024;
    OffMaps TM;
    std::memset(&TM, 0, sizeof TM);
    if (tma) {
        encode_tiled_fn enc = encoder();
        if (!enc) return cudaErrorNotSupported;
        const cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)A.K};
        const cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
        const cuuint32_t boxa[2] = {128, (cuuint32_t)KC}, boxb[2] = {(cuuint32_t)(A.NB / 2), (cuuint32_t)KC};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&TM.pu, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)Pu, dims, strides, boxa, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
            enc(&TM.pv, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)Pv, dims, strides, boxb, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    auto kern = tma ? offset_tc_kernel<true> : offset_tc_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // entries whose P_u point lies outside the row belong to no item: zero first
    e = cudaMemsetAsync(out, 0, (size_t)(2 * nh + 1) * N * sizeof(float), s);
    if (e != cudaSuccess) return e;
    const long long items = A.rows * A.ntx;
    const unsigned grid = (unsigned)std::min<long long>(items, sms);
    kern<<<grid, OT_THREADS, smem, s>>>(A, ST, TM);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
