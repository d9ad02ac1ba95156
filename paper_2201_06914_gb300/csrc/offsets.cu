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
//               This kernel (offset_tc_kernel) reads dense operands (rows N floats apart,
//               no alignment) with 4-byte loads into registers, two blocks of 32 in flight
//               per thread, and row-aligned operands whose band is too wide for the
//               MN-major kernel below (offset_mn_kernel, which stages row-aligned operands
//               by TMA and splits them in place);
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

__global__ void __launch_bounds__(OT_THREADS, 1) offset_tc_kernel(const OffArgs A, int ST)
{
    extern __shared__ uint8_t smem_raw[];
    // aligned by pointer arithmetic on the shared array (no integer round trip), so the
    // compiler keeps every access derived from it in the shared state space
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ uint64_t full[4], empty[4], accfull, accempty;
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
      {
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

// ---------------------------------------------------------------------------------------
// Row-aligned operands with MN-major tcgen05 operands (offset_mn_kernel)
// ---------------------------------------------------------------------------------------
// The staged FP32 tiles are the operands' own layout turned MN-major: a TMA box of P_u (128
// points x 64 k) or P_v (NBp / 2 points x 64 k, two boxes) lands with points contiguous
// and k rows one after the other.  Viewed in halves of 32 k, each half's bytes are exactly
// the bytes of that half's bf16 hi and lo operand atoms (64 points x 8 k, 128-byte swizzle,
// 1 KB each), so the split is done in place: every converter reads its share of a half into
// registers, the converters meet at a barrier, and each writes its hi and lo chunks.  With
// no separate staging area, two full stages fit, so a chunk's copies land while the
// previous chunk is converted and multiplied:
//   warp 12      producer: three tiled TMA copies per 64-k chunk into stage j mod 2 once
//                the MMAs of chunk j - 2 have released it;
//   warps 0-7    converters: per half, read (k, 8 points) units, zero the points outside
//                the x-row, barrier, write hi / lo;
//   warps 8-11   epilogue as in offset_tc_kernel; lane 0 of warp 8 issues the MMAs with
//                MN-major ("transposed") A and B descriptors.
// Atom addresses (bytes from the stage; kg = k / 8 within the chunk, mi / ni = point / 64,
// hl = 0 for hi, 1 for lo):
//   A: kg * 4096 + hl * 2048 + mi * 1024            (FP32 rows of 512 B: k row at 512 k)
//   B: 32768 + hl * 256 NBh + kg * 16 NBp + ni * 1024 (box hl's FP32 rows of 4 NBh bytes)
// so half h of A covers [16384 h, +16384) and half h of box b covers 32768 + 256 NBh b +
// [128 NBh h, +128 NBh) in both views.
constexpr int MN_THREADS = 416;   // warps 0-7 converters, 8-11 epilogue + MMA issue, 12 producer
constexpr int MN_WPROD = 12;
constexpr int MN_UNITS = 7;       // (k, 8-point) units per converter thread and half (NBp <= 320)

__host__ __device__ inline int mn_nbp(int NB) { return (NB + 63) / 64 * 64; }
__host__ __device__ inline uint32_t mn_stage_bytes(int NBp) { return 32768u + (uint32_t)NBp * 256u; }

// MN-major operand, 128-byte swizzle: atoms of 64 elements (along M or N) x 8 k; LBO = bytes
// between atoms along M / N, SBO = bytes between 8-k groups.
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__global__ void __maxnreg__(128) offset_mn_kernel(const OffArgs A, const __grid_constant__ OffMaps TM)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // a shared pointer
    __shared__ uint64_t fbar[2], full[2], empty[2], accfull, accempty;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NBp = mn_nbp(A.NB), NBh = NBp / 2;
    const uint32_t SBst = mn_stage_bytes(NBp);
    const uint32_t ncols = NBp > 256 ? 512 : 256;
    const long long nitems = A.rows * A.ntx;
    const int nch = (A.K + KC - 1) / KC;
    const long long myitems = ((long long)nitems - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const long long total = myitems * nch;   // chunks of this CTA

    if (tid == 0) {
        for (int s = 0; s < 2; s++) {
            mbar_init(&fbar[s], 1);
            mbar_init(&full[s], OCONV);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&accfull, 1);
        mbar_init(&accempty, 128);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == OW_EPI) tmem_alloc(&tmem_holder, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    auto stage_ptr = [&](int s) { return smem + (size_t)s * SBst; };

    if (warp == MN_WPROD) {
        // ---------------- producer ----------------
        if (lane == 0) {
            long long issued = -1;
            for (long long j = 0; j < total; j++) {
                const int s = (int)(j & 1);
                if (!mbar_wait_abortable(&empty[s], (uint32_t)((j >> 1) & 1) ^ 1u, &abort_flag)) break;
                const long long item = blockIdx.x + (j / nch) * (long long)gridDim.x;
                const int c = (int)(j % nch);
                const long long row = item / A.ntx;
                const int a0 = (int)(item - row * A.ntx) * 128;
                const int xa = (int)(row * A.XP) + a0, xb = xa - A.boff;
                uint8_t *st = stage_ptr(s);
                mbar_arrive_expect_tx(&fbar[s], SBst);
                off_tma_2d(st, &TM.pu, xa, c * KC, &fbar[s]);
                off_tma_2d(st + 32768, &TM.pv, xb, c * KC, &fbar[s]);
                off_tma_2d(st + 32768 + (size_t)NBh * 256, &TM.pv, xb + NBh, c * KC, &fbar[s]);
                issued = j;
            }
            // after an abort: let the copies still in flight land before the block exits
            if (issued >= 0 && abort_flag) {
                mbar_wait_bounded(&fbar[issued & 1], (uint32_t)((issued >> 1) & 1));
                if (issued >= 1) mbar_wait_bounded(&fbar[(issued - 1) & 1], (uint32_t)(((issued - 1) >> 1) & 1));
            }
        }
    } else if (warp < OW_EPI) {
        // ---------------- converters ----------------
        // Unit u < 512: A, k row u / 16 of the half, points 8 (u % 16) .. +7; u >= 512: box
        // b of B, k row and 8-point group from the remainder.  Offsets (bytes from the stage)
        // of a unit in half 0; half 1 adds HA (A) or HB (B) to both the FP32 source and the
        // atom destination, which is what makes the split in place.
        const int gB = NBh / 8;                       // 8-point groups per B box row
        const int nA = 32 * 16, nU = nA + 2 * 32 * gB;
        const uint32_t HA = 16384u, HB = 128u * (uint32_t)NBh, LOB = 256u * (uint32_t)NBh;
        uint32_t src[MN_UNITS], dst[MN_UNITS];
        int xr[MN_UNITS];   // first point's x relative to a0 (A) or b0 (B); INT_MIN: no unit
        bool isb[MN_UNITS];
#pragma unroll
        for (int i = 0; i < MN_UNITS; i++) {
            const int u = tid + OCONV * i;
            xr[i] = -0x40000000;
            isb[i] = false;
            src[i] = dst[i] = 0;
            if (u < nA) {
                const int k = u >> 4, p = (u & 15) * 8;
                src[i] = (uint32_t)(k * 512 + p * 4);
                dst[i] = (uint32_t)((k >> 3) * 4096 + (p >> 6) * 1024 + (k & 7) * 128 + ((((p & 63) >> 3) ^ (k & 7)) << 4));
                xr[i] = p;
            } else if (u < nU) {
                const int v = u - nA, b = v / (32 * gB), rm = v - b * 32 * gB;
                const int k = rm / gB, pb = (rm - k * gB) * 8, p = b * NBh + pb;
                src[i] = 32768u + (uint32_t)(b * NBh * 256 + (k * NBh + pb) * 4);
                dst[i] = 32768u + (uint32_t)((k >> 3) * NBp * 16 + (p >> 6) * 1024 + (k & 7) * 128 +
                                             ((((p & 63) >> 3) ^ (k & 7)) << 4));
                xr[i] = p;
                isb[i] = true;
            }
        }
        for (long long j = 0; j < total; j++) {
            const int s = (int)(j & 1);
            const long long item = blockIdx.x + (j / nch) * (long long)gridDim.x;
            const long long row = item / A.ntx;
            const int a0 = (int)(item - row * A.ntx) * 128, b0 = a0 - A.boff;
            const bool got = mbar_wait_abortable(&fbar[s], (uint32_t)((j >> 1) & 1), &abort_flag);
            if (bar_any<1, OCONV>(!got)) break;
            const uint32_t st = smem_u32(stage_ptr(s));
#pragma unroll
            for (int h = 0; h < 2; h++) {
                float v[MN_UNITS][8];
#pragma unroll
                for (int i = 0; i < MN_UNITS; i++) {
                    if (xr[i] == -0x40000000) continue;
                    const uint32_t a = st + src[i] + (h ? (isb[i] ? HB : HA) : 0u);
                    float4 q0, q1;
                    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                                 : "=f"(q0.x), "=f"(q0.y), "=f"(q0.z), "=f"(q0.w) : "r"(a));
                    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                                 : "=f"(q1.x), "=f"(q1.y), "=f"(q1.z), "=f"(q1.w) : "r"(a + 16));
                    v[i][0] = q0.x; v[i][1] = q0.y; v[i][2] = q0.z; v[i][3] = q0.w;
                    v[i][4] = q1.x; v[i][5] = q1.y; v[i][6] = q1.z; v[i][7] = q1.w;
                    const int x = (isb[i] ? b0 : a0) + xr[i];
#pragma unroll
                    for (int e = 0; e < 8; e++)
                        if (x + e < 0 || x + e >= A.NX) v[i][e] = 0.f;   // outside the x-row
                }
                asm volatile("bar.sync 3, %0;" ::"n"(OCONV) : "memory");   // half h read by all
#pragma unroll
                for (int i = 0; i < MN_UNITS; i++) {
                    if (xr[i] == -0x40000000) continue;
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) split_bf16x2(v[i][2 * e], v[i][2 * e + 1], hi[e], lo[e]);
                    const uint32_t a = st + dst[i] + (h ? (isb[i] ? HB : HA) : 0u);
                    const uint32_t al = a + (isb[i] ? LOB : 2048u);
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(hi[0]), "r"(hi[1]),
                                 "r"(hi[2]), "r"(hi[3]) : "memory");
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(al), "r"(lo[0]), "r"(lo[1]),
                                 "r"(lo[2]), "r"(lo[3]) : "memory");
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&full[s]);
        }
    } else {
        // ---------------- epilogue (warps 8-11), MMA issue in lane 0 of warp 8 ----------------
        const int ew = warp - OW_EPI;
        const int N1 = NBp < 256 ? NBp : 256, N2 = NBp - N1;
        constexpr uint32_t MNMAJ = (1u << 15) | (1u << 16);   // A and B MN-major
        const uint32_t id1 = idesc_bf16_f32(128, N1) | MNMAJ, id2 = N2 > 0 ? (idesc_bf16_f32(128, N2) | MNMAJ) : 0u;
        const uint32_t sbo_b = 16u * (uint32_t)NBp, lob = 256u * (uint32_t)NBh;
        long long gm = 0;   // chunks consumed by the MMA issue
        const int al = ew * 32 + lane;   // a - a0 of this lane
        const int c_lo = std::max(0, ew * 32 + A.boff - 2 * A.nh) & ~15;
        const int c_hi = std::min(A.NB, ew * 32 + 32 + A.boff + 2 * A.nh);
        uint32_t jt = 0;
        for (long long item = blockIdx.x; item < nitems; item += gridDim.x, jt++) {
            const long long row = item / A.ntx;
            const int a0 = (int)(item - row * A.ntx) * 128;
            if (ew == 0) {
                if (lane == 0 && mbar_wait_abortable(&accempty, (jt & 1) ^ 1, &abort_flag)) {
                    tc_fence_after();
                    for (int c = 0; c < nch; c++, gm++) {
                        const int s = (int)(gm & 1);
                        if (!mbar_wait_abortable(&full[s], (uint32_t)((gm >> 1) & 1), &abort_flag)) break;
                        tc_fence_after();
                        const uint32_t ab = smem_u32(stage_ptr(s)), bb = ab + 32768u;
#pragma unroll
                        for (int ks = 0; ks < KC / 16; ks++) {   // 16 k = two 8-k groups
                            const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
                            const uint32_t ak = ab + (uint32_t)(2 * ks) * 4096u, bk = bb + (uint32_t)(2 * ks) * sbo_b;
                            const uint64_t dah = sdesc_mn_sw128(ak, 1024u, 4096u), dal = sdesc_mn_sw128(ak + 2048u, 1024u, 4096u);
                            {
                                const uint64_t dbh = sdesc_mn_sw128(bk, 1024u, sbo_b), dbl = sdesc_mn_sw128(bk + lob, 1024u, sbo_b);
                                umma_bf16(tmem, dah, dbh, id1, acc0);
                                umma_bf16(tmem, dal, dbh, id1, 1u);
                                umma_bf16(tmem, dah, dbl, id1, 1u);
                                umma_bf16(tmem, dal, dbl, id1, 1u);
                            }
                            if (N2 > 0) {
                                const uint32_t o2 = (uint32_t)(N1 / 64) * 1024u;
                                const uint64_t dbh = sdesc_mn_sw128(bk + o2, 1024u, sbo_b);
                                const uint64_t dbl = sdesc_mn_sw128(bk + lob + o2, 1024u, sbo_b);
                                const uint32_t t2 = tmem + (uint32_t)N1;
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
            const bool ok = mbar_wait_abortable(&accfull, jt & 1, &abort_flag);
            if (bar_any<2, 128>(!ok)) break;
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(ew * 32) << 16);
            float *orow = A.out + row * A.NX;
            for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
                uint32_t r16[16];
                tmem_ld16(taddr + (uint32_t)c0, r16);
#pragma unroll
                for (int q = 0; q < 16; q++) {
                    const int d = al + A.boff - (c0 + q);   // a - b
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
    const size_t avail = 227 * 1024 - 1024;
    // entries whose P_u point lies outside the row belong to no item: zero first
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)(2 * nh + 1) * N * sizeof(float), s);
    if (e != cudaSuccess) return e;
    const long long items = A.rows * A.ntx;
    const unsigned grid = (unsigned)std::min<long long>(items, sms);
    // aligned rows: MN-major operands split in place, two stages, when both fit (NB rounded
    // up to 64 <= 320: nh <= 48); wider bands read the aligned rows with the register loads
    // of the dense path
    const int NBp = mn_nbp(A.NB);
    const uint32_t SBm = mn_stage_bytes(NBp);
    if (aligned && 2 * (size_t)SBm <= avail) {
        encode_tiled_fn enc = encoder();
        if (!enc) return cudaErrorNotSupported;
        OffMaps TM;
        std::memset(&TM, 0, sizeof TM);
        const cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)A.K};
        const cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
        const cuuint32_t boxa[2] = {128, (cuuint32_t)KC}, boxb[2] = {(cuuint32_t)(NBp / 2), (cuuint32_t)KC};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&TM.pu, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)Pu, dims, strides, boxa, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
            enc(&TM.pv, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)Pv, dims, strides, boxb, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
        const size_t smem = 2 * (size_t)SBm + 1024;
        e = cudaFuncSetAttribute(offset_mn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        offset_mn_kernel<<<grid, MN_THREADS, smem, s>>>(A, TM);
    } else {
        const uint32_t SB = off_stage_bytes(A.NB);
        const int ST = (int)std::min<size_t>(4, avail / SB);
        if (ST < 1) return cudaErrorInvalidValue;
        const size_t smem = (size_t)ST * SB + 1024;
        e = cudaFuncSetAttribute(offset_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        offset_tc_kernel<<<grid, OT_THREADS, smem, s>>>(A, ST);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
