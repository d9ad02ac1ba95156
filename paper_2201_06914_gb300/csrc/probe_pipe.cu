// Pipelined probe accumulation on the tensor cores (Eq. 3), the hot-path version of
// probe_gemm.cu.  For every shot and every 128-point tile of the grid:
//   P[i][x] += scale * sum_{t < cnt} A[t][x] * Q[t0 + t][i]
// where A is read from the time-step ring (forward: u_tt rebuilt from two consecutive
// stored increments; adjoint: the adjoint wavefield itself).
//
// One persistent CTA per SM runs a warp-specialised pipeline over its (shot, tile) items:
//   warp 12    producer: per 64-step chunk, one or two tiled TMA copies of the 64 (or 65)
//              ring rows of the tile plus the pre-swizzled probe image(s) (bf16 hi, and lo
//              unless the probes are exact bfloat16 values) into a stage of shared memory,
//              completing on the stage's `full` mbarrier;
//   warps 0-7  converters: one grid point and half of the chunk's steps per thread,
//              FP32 -> u_tt (or v) -> bfloat16 hi + lo, written in the K-major
//              128-byte-swizzled layout tcgen05 reads;
//   warp 13    MMA issuer (one thread): 2 or 4 bf16 products per 16-step k-slice into the
//              TMEM accumulator (double-buffered up to 256 probes; one of 512 columns,
//              each product two MMAs, above); commits release the stage and, after the
//              last chunk of an item, hand the accumulator to the epilogue;
//   warps 8-11 epilogue: tcgen05.ld of the accumulator into shared-memory slices that a
//              TMA tensor store (first block) or reduce-add writes to P (the randomized
//              imaging condition runs afterwards, probe_dot_kernel / probe_dot4_kernel).
// Every wait is bounded; a wait that gives up raises the kernel error flag and all roles
// leave their loops, the TMEM is freed and the kernel returns.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "wp_internal.cuh"

namespace wp {

namespace {

constexpr int PIPE_THREADS = 448;
constexpr int NCONV = 256;                // converter threads (warps 0-7)
constexpr int WEPI = 8, WPROD = 12, WMMA = 13;
constexpr int CH = 64;                    // time steps per chunk
constexpr int MAXCH = 8;                  // chunks per block covered by tensor maps (Tb <= 512)
constexpr int PSL = 64;                   // probes per epilogue slice (TMA box rows), r_pad <= 16

// Probes per epilogue slice for r_pad.  The staging of two slices shares shared memory with
// the pipeline stages (41 KiB a stage at 32 probes, 49 KiB at 64, 65 KiB at 128, 97 KiB at
// 256): two 64-probe slices (64 KiB) leave room for 3, 3, 2 and 1 stages, two 16-probe
// slices (16 KiB) for 4 (the most the kernel uses), 4, 3 and 2.  At 16 probes four stages
// fit either way.  Above 256 probes the single accumulator waits for the epilogue to drain
// it, so fewer, taller slices pay: 32-probe slices (32 KiB) keep the two stages without the
// lo image up to 496 probes (at 448: 25.5 instead of 28.0 ms per 512-step block of 32
// shots); at 512 only 16-probe slices leave room for two.
__host__ __device__ constexpr int psl_of(int r_pad)
{
    return r_pad <= 16 ? PSL : (r_pad > 256 && r_pad <= 496) ? 32 : 16;
}

// Tiled TMA descriptors of the ring for one launch.  Chunk c of every item covers the ring
// slots [s0_c, s0_c + rows_c) modulo nslots, the same for all items of the launch; piece 0
// is the run of slots before the ring wraps, piece 1 the run after it (from slot 0).  The
// tensor is [shot][slot][point] with the tile's 128 points as the box's inner extent, so
// one chunk is one or two copies instead of one per slot.
struct PipeMaps {
    CUtensorMap map[MAXCH][2];
    CUtensorMap pmap;   // P as [shot][probe][point]: boxes of 128 points x 64 probes
    int slot[MAXCH][2];
    int rows[MAXCH][2];
    int use;
};

// TMA tensor store / reduce-add of a [64][128] float box from shared memory into P.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void tma_reduce_add_3d(const CUtensorMap *map, const void *src, int x, int y, int z)
{
    asm volatile("cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Named barrier over the 128 epilogue threads; the OR form returns whether any of them
// failed its wait, so all leave their loop together.
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 2, 128;" ::: "memory"); }
__device__ __forceinline__ bool epi_any(bool failed)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred q, p;\n\t"
                 "setp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.or.pred p, 2, 128, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r) : "r"((uint32_t)failed) : "memory");
    return r != 0;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
constexpr uint32_t A32_BYTES = 33792;     // 65 rows x 512 B, rounded to 1 KiB

__host__ __device__ inline uint32_t pipe_cols(int r_pad)
{
    uint32_t c = 32;
    while (c < (uint32_t)r_pad) c <<= 1;
    return c;
}

// Stage = [A region: 65 FP32 ring rows, overwritten in place by the bf16 hi/lo operand
//          (2 x 16 KiB) once all converter threads have read their column]
//         [probe image hi][probe image lo, only when the probes have a non-zero lo part]
__host__ __device__ inline uint32_t stage_bytes(int r_pad, bool lo)
{
    return A32_BYTES + (lo ? 2u : 1u) * (uint32_t)r_pad * 128u;
}

// Shared-memory plan of one launch.  Whether the probes' lo image is staged is known only on
// the device (the flag launch_probe_images writes), so the host sizes both plans and the
// kernel takes the one the flag selects; the epilogue staging sits after the larger one.
// Without the lo image a stage is smaller, which above 256 probes makes room for two.
struct PipePlan {
    uint32_t sb[2];     // stage bytes without / with the lo image
    int st[2];          // stages (1..MAXST) without / with the lo image
    uint32_t stg_off;   // byte offset of the epilogue staging
};
constexpr int MAXST = 4;

// Named barrier over the 256 converter threads that also returns, to every one of them,
// whether any of them failed its wait: the converters leave their loops together, so no
// thread is left waiting at the barrier for one that has gone.
__device__ __forceinline__ bool converters_any(bool failed)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred q, p;\n\t"
                 "setp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.or.pred p, 1, 256, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r) : "r"((uint32_t)failed) : "memory");
    return r != 0;
}

// try_wait that lets the hardware suspend the thread for up to `ns` nanoseconds (it wakes
// as soon as the phase completes), so waiting roles do not spin on the issue slots the
// converters and the epilogue need.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    const long long t0 = clock64();
    while (!mbar_try_wait_sleep(bar, parity, 100000u)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > (1ll << 31)) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// p / d for the ring's point index; 32-bit division when the ring rows are below 2^31 points
__device__ __forceinline__ long long div_pts(long long p, int d, bool small)
{
    return small ? (long long)((uint32_t)p / (uint32_t)d) : p / d;
}

// (a, b) -> bf16 pairs hi = rn(a, b) and lo = rn(a - hi_a, b - hi_b), a in the low halves
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - __low2float(h), b - __high2float(h));
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

}  // namespace

// RB: a compile-time bound on r_pad (16, 32, 64, 128, 256 or 512) so the epilogue's column
// loops unroll with constant column offsets; PS: probes per epilogue slice (psl_of).  Up to
// 256 probes the accumulator is double-buffered in tensor memory (the epilogue of one item
// overlaps the MMAs of the next); above, one accumulator takes all 512 columns and each
// product is two MMAs (N = 256 and r_pad - 256, the largest N of one instruction being 256),
// so the ring is read once for up to 512 probes.
template <int RB, int PS>
__global__ void __launch_bounds__(PIPE_THREADS, 1) probe_pipe_kernel(const PipeArgs A, const PipePlan PL, int nshots,
                                                                     const __grid_constant__ PipeMaps TM)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);   // stays a shared pointer
    __shared__ uint64_t full[MAXST], empty[MAXST], aready[MAXST], accfull[2], accempty[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // probes that are exact bfloat16 values (Rademacher +-1) have an all-zero lo part: its
    // image is not staged and its two products are skipped (the flag is written before this
    // launch, so every thread reads the same value)
    const bool qlo = !A.qlo_nz || *(volatile const int *)A.qlo_nz != 0;
    const uint32_t SB = qlo ? PL.sb[1] : PL.sb[0];   // selects, not an indexed parameter array
    const int ST = qlo ? PL.st[1] : PL.st[0];
    const uint32_t ncols = pipe_cols(A.r_pad);
    const uint32_t nacc = ncols <= 256 ? 2u : 1u;   // accumulators in tensor memory
    const int nitems = A.ntiles * nshots;
    const bool small = A.Np + 128 < (1LL << 31);
    const int nch = (A.cnt + CH - 1) / CH;

    if (tid == 0) {
        for (int s = 0; s < ST; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&aready[s], NCONV);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], 128);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == WMMA) tmem_alloc(&tmem_holder, nacc * ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;

    auto stage_ptr = [&](int s) { return smem + (size_t)s * SB; };

    if (warp == WPROD) {
        // ---------------- producer ----------------
        uint32_t g = 0;
        for (int item = blockIdx.x; item < nitems && !abort_flag; item += gridDim.x) {
            const int shot = item / A.ntiles, tile = item % A.ntiles;
            const float *ring = A.ring + (long long)shot * A.ring_ss + (long long)tile * 128;
            const size_t img_bytes = (size_t)A.r_pad * 128;
            for (int c = 0; c < nch; c++, g++) {
                const int s = g % ST;
                const uint32_t ph = (g / ST) & 1;
                if (!wait_bar(&empty[s], ph ^ 1, &abort_flag)) break;
                const int need = A.cnt - c * CH;
                const int rows = A.mode ? min(CH + 1, need + 1) : min(CH, need);
                uint8_t *st = stage_ptr(s);
                if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)(rows * 512 + (qlo ? 2 : 1) * img_bytes));
                __syncwarp();
                if (TM.use) {
                    if (lane == 0) {
                        tma_load_3d(st, &TM.map[c][0], tile * 128, TM.slot[c][0], shot, &full[s]);
                        if (TM.rows[c][1] > 0)
                            tma_load_3d(st + (size_t)TM.rows[c][0] * 512, &TM.map[c][1], tile * 128, 0,
                                        shot, &full[s]);
                    }
                } else {
                    const int s0 = (A.slot0 + c * CH) % A.nslots;
                    for (int t = lane; t < rows; t += 32) {
                        int slot = s0 + t;
                        while (slot >= A.nslots) slot -= A.nslots;
                        bulk_g2s(st + (size_t)t * 512, ring + (long long)slot * A.sstride, 512, &full[s]);
                    }
                }
                if (lane == 0) {
                    const long long im = ((long long)(shot / A.img_div) * A.nblocks + A.blk) * A.ncb + c;
                    const uint8_t *hi = (const uint8_t *)(A.img_hi + im * A.img_ld);
                    const uint8_t *lo = (const uint8_t *)(A.img_lo + im * A.img_ld);
                    bulk_g2s(st + A32_BYTES, hi, (uint32_t)img_bytes, &full[s]);
                    if (qlo) bulk_g2s(st + A32_BYTES + img_bytes, lo, (uint32_t)img_bytes, &full[s]);
                }
                __syncwarp();
            }
        }
    } else if (warp == WMMA) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            // probes [0, n1) and, above 256, [256, 256 + n2) (image rows, accumulator columns)
            const int n1 = A.r_pad < 256 ? A.r_pad : 256, n2 = A.r_pad - n1;
            const uint32_t idesc = idesc_bf16_f32(128, n1);
            const uint32_t idesc2 = idesc_bf16_f32(128, n2 > 0 ? n2 : 16);
            const uint32_t img_bytes = (uint32_t)A.r_pad * 128;
            uint32_t g = 0, j = 0;
            for (int item = blockIdx.x; item < nitems && !abort_flag; item += gridDim.x, j++) {
                const uint32_t ab = nacc == 2 ? (j & 1) : 0u, aph = nacc == 2 ? ((j >> 1) & 1) : (j & 1);
                if (!wait_bar(&accempty[ab], aph ^ 1, &abort_flag)) break;
                tc_fence_after();
                const uint32_t dt = tmem + ab * ncols;
                bool ok = true;
                for (int c = 0; c < nch; c++, g++) {
                    const int s = g % ST;
                    if (!wait_bar(&aready[s], (g / ST) & 1, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(stage_ptr(s));
                    const uint32_t bh = base + A32_BYTES, bl = bh + img_bytes;
                    const uint32_t ah = base, al = ah + 16384;
#pragma unroll
                    for (int k = 0; k < CH / 16; k++) {
                        const uint32_t ko = (uint32_t)k * 32u;
                        const uint64_t dah = sdesc_k_sw128(ah + ko), dal = sdesc_k_sw128(al + ko);
                        const uint64_t dbh = sdesc_k_sw128(bh + ko), dbl = sdesc_k_sw128(bl + ko);
                        const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
                        umma_bf16(dt, dah, dbh, idesc, acc);
                        umma_bf16(dt, dal, dbh, idesc, 1u);
                        if (qlo) {
                            umma_bf16(dt, dah, dbl, idesc, 1u);
                            umma_bf16(dt, dal, dbl, idesc, 1u);
                        }
                        if (RB > 256) {
                            // rows 256.. of the images start 256 x 128 B further (a whole
                            // number of 1 KiB swizzle atoms); columns 256.. of the accumulator
                            const uint64_t dbh2 = sdesc_k_sw128(bh + 32768u + ko), dbl2 = sdesc_k_sw128(bl + 32768u + ko);
                            umma_bf16(dt + 256u, dah, dbh2, idesc2, acc);
                            umma_bf16(dt + 256u, dal, dbh2, idesc2, 1u);
                            if (qlo) {
                                umma_bf16(dt + 256u, dah, dbl2, idesc2, 1u);
                                umma_bf16(dt + 256u, dal, dbl2, idesc2, 1u);
                            }
                        }
                    }
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&accfull[ab]);
            }
        }
    } else if (warp < WEPI) {
        // ---------------- converters ----------------
        const int m = tid & 127, half = tid >> 7;   // point, steps [32 half, 32 half + 32)
        uint32_t g = 0;
        // No early exit on the abort flag here: a failed wait is voted on by all converters
        for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
            const int tile = item % A.ntiles;
            const long long p = (long long)tile * 128 + m;
            const long long prow = div_pts(p, A.NXp, small);
            const bool valid = p < A.Np && (int)(p - prow * A.NXp) < A.NX;
            float cp = 1.f, cm = 1.f;
            if (A.mode == 1 && valid) {
                const int x = (int)(p - prow * A.NXp);
                const int z = (int)div_pts(prow, A.G.NY, small), y = (int)(prow - (long long)z * A.G.NY);
                const float sd = damp_at(A.G, x, y, z);
                cp = 1.f + sd;
                cm = 1.f - sd;
            }
            bool ok = true;
            for (int c = 0; c < nch; c++, g++) {
                const int s = g % ST;
                const bool got = wait_bar(&full[s], (g / ST) & 1, &abort_flag);
                uint8_t *st = stage_ptr(s);
                const float *a32 = (const float *)st;
                uint8_t *ah = st;            // the operand overwrites the FP32 rows in place
                uint8_t *al = ah + 16384;
                const int need = A.cnt - c * CH - half * (CH / 2);   // valid steps of this half
                const bool rd = valid && got;
                const float *col = a32 + half * (CH / 2) * 128 + m;
                float v[CH / 2];
                if (A.mode == 0) {
#pragma unroll
                    for (int t = 0; t < CH / 2; t++) v[t] = (rd && t < need) ? col[t * 128] : 0.f;
                } else {
                    float prev = (rd && need > 0) ? col[0] : 0.f;
#pragma unroll
                    for (int t = 0; t < CH / 2; t++) {
                        const bool in = rd && t < need;
                        const float nx = in ? col[(t + 1) * 128] : 0.f;
                        v[t] = in ? cp * nx - cm * prev : 0.f;
                        prev = nx;
                    }
                }
                // every converter has read its FP32 column before any operand byte is written
                if (converters_any(!got)) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int c4 = 0; c4 < 4; c4++) {
                    const int cc = half * 4 + c4;   // 16-byte chunk = 8 steps of the row
                    const uint32_t off = (uint32_t)m * 128u + ((uint32_t)(cc ^ (m & 7)) << 4);
                    const float *x = v + c4 * 8;
                    uint4 h, l;
                    split2(x[0], x[1], h.x, l.x);
                    split2(x[2], x[3], h.y, l.y);
                    split2(x[4], x[5], h.z, l.z);
                    split2(x[6], x[7], h.w, l.w);
                    *(uint4 *)(ah + off) = h;
                    *(uint4 *)(al + off) = l;
                }
                fence_proxy_async_smem();
                mbar_arrive(&aready[s]);
            }
            if (!ok) break;
        }
    } else {
        // ---------------- epilogue (warps 8-11) ----------------
        // The accumulator of an item goes to P in slices of PS probes: tcgen05.ld, scale,
        // shared-memory staging [PS][128] (two buffers), then one TMA tensor store (first
        // block of a pass) or reduce-add (later blocks) per slice: P is never read by an SM.
        const int e = tid - NCONV, ew = warp - WEPI;
        float *stg0 = (float *)(smem + PL.stg_off);   // [2][PS][128]
        int sbuf = 0;
        uint32_t j = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x, j++) {
            const int shot = item / A.ntiles, tile = item % A.ntiles;
            const uint32_t ab = nacc == 2 ? (j & 1) : 0u, aph = nacc == 2 ? ((j >> 1) & 1) : (j & 1);
            const bool ok = wait_bar(&accfull[ab], aph, &abort_flag);
            if (epi_any(!ok)) break;
            tc_fence_after();
            const uint32_t taddr = tmem + ab * ncols + ((uint32_t)(ew * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < RB; c0 += PS) {
                if (c0 < A.r_pad) {
                    float *stg = stg0 + (size_t)sbuf * PS * 128;
                    if (e == 0) bulk_wait_read<1>();   // the TMA op that last read this buffer is done
                    epi_bar();
#pragma unroll
                    for (int c = c0; c < c0 + PS && c < RB; c += 16) {
                        if (c < A.r_pad) {
                            uint32_t r16[16];
                            tmem_ld16(taddr + (uint32_t)c, r16);
#pragma unroll
                            for (int q = 0; q < 16; q++)
                                stg[(c - c0 + q) * 128 + e] = A.scale * __uint_as_float(r16[q]);
                        }
                    }
                    fence_proxy_async_smem();
                    epi_bar();
                    if (e == 0) {
                        if (A.p_zero) tma_store_3d(&TM.pmap, stg, tile * 128, c0, shot);
                        else tma_reduce_add_3d(&TM.pmap, stg, tile * 128, c0, shot);
                        bulk_commit();
                    }
                    sbuf ^= 1;
                }
            }
            tc_fence_before();
            mbar_arrive(&accempty[ab]);
        }
        if (e == 0) bulk_wait_all();   // every store has read shared memory and completed
    }

    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(A.err, 2);
    if (warp == WMMA) {
        tc_fence_after();
        tmem_dealloc(tmem, nacc * ncols);
    }
}

static int g_num_sms = 0;

// cuTensorMapEncodeTiled from the driver (no link-time dependency on libcuda), or nullptr.
encode_tiled_fn encoder()
{
    static encode_tiled_fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (encode_tiled_fn)p;
    }
    return fn;
}

// Ring maps for the chunks of this launch; use = 0 (per-slot bulk copies) when a map cannot
// be encoded, e.g. for a caller's ring whose rows are not 16-byte multiples.
static PipeMaps ring_maps(const PipeArgs &A, int nshots)
{
    PipeMaps TM;
    memset(&TM, 0, sizeof TM);
    const int nch = (A.cnt + CH - 1) / CH;
    encode_tiled_fn enc = encoder();
    if (!enc || nch > MAXCH || ((uintptr_t)A.ring & 15)) return TM;
    const cuuint64_t dims[3] = {(cuuint64_t)A.Np, (cuuint64_t)A.nslots, (cuuint64_t)nshots};
    const cuuint64_t strides[2] = {(cuuint64_t)A.sstride * 4, (cuuint64_t)A.ring_ss * 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int c = 0; c < nch; c++) {
        const int need = A.cnt - c * CH;
        const int rows = A.mode ? std::min(CH + 1, need + 1) : std::min(CH, need);
        const int s0 = (A.slot0 + c * CH) % A.nslots;
        const int r0 = std::min(rows, A.nslots - s0), r1 = rows - r0;
        if (r1 > A.nslots) return TM;   // ring shorter than a chunk: per-slot copies
        const int pr[2] = {r0, r1};
        for (int k = 0; k < 2; k++) {
            TM.slot[c][k] = k ? 0 : s0;
            TM.rows[c][k] = pr[k];
            if (pr[k] == 0) continue;
            const cuuint32_t box[3] = {128, (cuuint32_t)pr[k], 1};
            if (enc(&TM.map[c][k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)A.ring, dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
                TM.use = 0;
                return TM;
            }
        }
    }
    TM.use = 1;
    return TM;
}

// Tensor map of P ([shot][probe][point], rows P_pitch floats apart) for the epilogue.
static bool p_map(const PipeArgs &A, int nshots, int psl, CUtensorMap *map)
{
    encode_tiled_fn enc = encoder();
    if (!enc || ((uintptr_t)A.P & 15) || (A.P_pitch & 3) || (A.P_ss & 3)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)A.P_pitch, (cuuint64_t)A.r, (cuuint64_t)nshots};
    const cuuint64_t strides[2] = {(cuuint64_t)A.P_pitch * 4, (cuuint64_t)A.P_ss * 4};
    const cuuint32_t box[3] = {128, (cuuint32_t)psl, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)A.P, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static cudaError_t launch_probe_pipe_slice(const PipeArgs &A, int nshots, cudaStream_t s);

// Up to 512 probes (the tensor memory's columns) the ring is read once.  More would run one
// launch per slice of 512 probes: a slice reads rows [i0, i0 + 512) of the probe images (a
// multiple of 8 rows, so the 128-byte swizzle pattern is unchanged), writes rows [i0, ..) of
// P and reads the ring again.
constexpr int PIPE_MAX_R = 512;
cudaError_t launch_probe_pipe(const PipeArgs &A, int nshots, cudaStream_t s)
{
    if (A.r <= PIPE_MAX_R) return launch_probe_pipe_slice(A, nshots, s);
    for (int i0 = 0; i0 < A.r; i0 += PIPE_MAX_R) {
        PipeArgs B = A;
        B.r = std::min(PIPE_MAX_R, A.r - i0);
        B.r_pad = std::min(PIPE_MAX_R, A.r_pad - i0);
        B.P = A.P + (long long)i0 * A.P_pitch;
        B.img_hi = A.img_hi + (long long)i0 * 64;
        B.img_lo = A.img_lo + (long long)i0 * 64;
        const cudaError_t e = launch_probe_pipe_slice(B, nshots, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t launch_probe_pipe_slice(const PipeArgs &A, int nshots, cudaStream_t s)
{
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    if (A.r_pad < 16 || A.r_pad > PIPE_MAX_R || A.r_pad % 16) return cudaErrorInvalidValue;
    const int rb = A.r_pad <= 16 ? 16 : A.r_pad <= 32 ? 32 : A.r_pad <= 64 ? 64 : A.r_pad <= 128 ? 128
                 : A.r_pad <= 256 ? 256 : 512;
    const int psl = psl_of(A.r_pad);
    const size_t pbytes = (size_t)2 * psl * 128 * 4;   // epilogue staging of P (two slices)
    const size_t avail = 227 * 1024 - 1024 - 256 - pbytes;
    PipePlan PL;
    for (int lo = 0; lo < 2; lo++) {
        PL.sb[lo] = stage_bytes(A.r_pad, lo != 0);
        PL.st[lo] = (int)std::min<size_t>(MAXST, avail / PL.sb[lo]);
        if (PL.st[lo] < 1) return cudaErrorInvalidValue;
    }
    // Deeper pipelines measured slower once P's traffic is large (4 instead of 3 stages at
    // 128 probes, 3 instead of 2 at 256: 5-6 % longer), so without the lo image the plan
    // keeps the stage count of the plan with it, except that it takes two stages where that
    // one has a single stage (above 256 probes).
    PL.st[0] = std::min(PL.st[0], std::max(PL.st[1], 2));
    PL.stg_off = std::max((uint32_t)PL.st[0] * PL.sb[0], (uint32_t)PL.st[1] * PL.sb[1]);
    const size_t smem = (size_t)PL.stg_off + pbytes + 1024;
    auto kern = rb == 16 ? probe_pipe_kernel<16, PSL> : rb == 32 ? probe_pipe_kernel<32, 16>
              : rb == 64 ? probe_pipe_kernel<64, 16> : rb == 128 ? probe_pipe_kernel<128, 16>
              : rb == 256 ? probe_pipe_kernel<256, 16>
              : psl == 32 ? probe_pipe_kernel<512, 32> : probe_pipe_kernel<512, 16>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long items = (long long)A.ntiles * nshots;
    if (items >= (1LL << 31)) return cudaErrorInvalidValue;
    dim3 grid((unsigned)std::min<long long>(items, g_num_sms));
    cudaEvent_t ev = prof_begin(PROF_GEMM, s);
    PipeMaps TM = ring_maps(A, nshots);
    if (A.ntiles * 128LL > A.P_pitch || !p_map(A, nshots, psl, &TM.pmap)) return cudaErrorInvalidValue;
    kern<<<grid, PIPE_THREADS, smem, s>>>(A, PL, nshots, TM);
    prof_end(PROF_GEMM, ev, s);
    count_launch();
    return cudaGetLastError();
}

// Swizzled probe images.  Image (shot, b, c) holds rows i < r_pad and 64 columns k, value
// Q[shot][t][i] for t = t_first + b*Tb + c*64 + k inside block b and below nt (else 0),
// split into bf16 hi and lo; byte offset of (i, k): i*128 + (((k/8) ^ (i%8)) * 16) + (k%8)*2.
__global__ void probe_image_kernel(const float *Q, int nt, int r, int r_pad, int t_first, int Tb,
                                   int nblocks, int ncb, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int *lo_nz)
{
    const long long im = blockIdx.x;
    const int i = blockIdx.y, k = threadIdx.x;
    const int c = (int)(im % ncb);
    const long long sb = im / ncb;
    const int b = (int)(sb % nblocks);
    const int shot = (int)(sb / nblocks);
    const int t = t_first + b * Tb + c * 64 + k;
    const int tend = min(t_first + (b + 1) * Tb, nt);
    float x = 0.f;
    if (i < r && c * 64 + k < Tb && t < tend) x = Q[((long long)shot * nt + t) * r + i];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    const long long base = im * (long long)r_pad * 64;
    const int off = i * 64 + (((k >> 3) ^ (i & 7)) << 3) + (k & 7);
    hi[base + off] = h;
    lo[base + off] = l;
    if (lo_nz && __bfloat162float(l) != 0.f) *lo_nz = 1;
}

cudaError_t launch_probe_images(const float *Q, int nshots, int nt, int r, int r_pad,
                                int t_first, int Tb, int nblocks, __nv_bfloat16 *hi,
                                __nv_bfloat16 *lo, int *lo_nz, cudaStream_t s)
{
    const int ncb = (Tb + 63) / 64;
    dim3 grid((unsigned)((long long)nshots * nblocks * ncb), r_pad);
    probe_image_kernel<<<grid, 64, 0, s>>>(Q, nt, r, r_pad, t_first, Tb, nblocks, ncb, hi, lo, lo_nz);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp

namespace wp {

// Randomized imaging condition (Eq. 3) summed over the shots:
//   g[u] = scale * sum_s sum_i P_u[s][i][.] * P_v[s][i][w(u)]
// with P_v in the row-aligned layout (rows of `pitch` floats, point w(u) at row pitch NXp)
// and P_u either dense ([shot][r][N], at u) or, with pu_aligned, row-aligned like P_v; one
// thread per grid point, shots and probes in a fixed order (deterministic).
__global__ void probe_dot_kernel(const float *__restrict__ Pu, bool pu_aligned, const float *__restrict__ Pv,
                                 long long N, int NX, int NXp, long long pitch, int r, int nshots, float scale,
                                 float *__restrict__ g)
{
    const long long apitch = pu_aligned ? pitch : N;
    for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < N;
         u += (long long)gridDim.x * blockDim.x) {
        const long long row = u / NX;
        const long long w = row * NXp + (u - row * NX);
        float acc = 0.f;
        for (int s = 0; s < nshots; s++) {
            const float *a = Pu + (long long)s * r * apitch + (pu_aligned ? w : u);
            const float *b = Pv + (long long)s * r * pitch + w;
            float part = 0.f;
#pragma unroll 8
            for (int i = 0; i < r; i++) part = fmaf(a[(long long)i * apitch], b[(long long)i * pitch], part);
            acc += part;
        }
        g[u] = scale * acc;
    }
}

// Both operands row-aligned: one thread per 4 consecutive points of a row (16-byte loads of
// both operands; rows of NXp points, a multiple of 4), the same per-point summation order
// as probe_dot_kernel, so the image is bitwise the same.
__global__ void probe_dot4_kernel(const float *__restrict__ Pu, const float *__restrict__ Pv, long long rows,
                                  int NX, int NXp, long long pitch, int r, int nshots, float scale,
                                  float *__restrict__ g)
{
    const int q4 = NXp / 4;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < rows * q4;
         t += (long long)gridDim.x * blockDim.x) {
        const long long row = t / q4;
        const int x = (int)(t - row * q4) * 4;
        const long long w = row * NXp + x;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int sh = 0; sh < nshots; sh++) {
            const float *a = Pu + (long long)sh * r * pitch + w;
            const float *b = Pv + (long long)sh * r * pitch + w;
            float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int i = 0; i < r; i++) {
                const float4 av = __ldg((const float4 *)(a + (long long)i * pitch));
                const float4 bv = __ldg((const float4 *)(b + (long long)i * pitch));
                part[0] = fmaf(av.x, bv.x, part[0]);
                part[1] = fmaf(av.y, bv.y, part[1]);
                part[2] = fmaf(av.z, bv.z, part[2]);
                part[3] = fmaf(av.w, bv.w, part[3]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) acc[j] += part[j];
        }
        float *gr = g + row * NX;
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (x + j < NX) gr[x + j] = scale * acc[j];
    }
}

cudaError_t launch_probe_dot(const float *Pu, bool pu_aligned, const float *Pv, long long N, int NX, int NXp,
                             long long pitch, int r, int nshots, float scale, float *g, cudaStream_t s)
{
    if (pu_aligned && (NXp & 3) == 0 && (pitch & 3) == 0 && !((uintptr_t)Pu & 15) && !((uintptr_t)Pv & 15)) {
        const long long rows = N / NX, work = rows * (NXp / 4);
        const long long blocks = std::min<long long>((work + 255) / 256, 152LL * 64);
        probe_dot4_kernel<<<(unsigned)blocks, 256, 0, s>>>(Pu, Pv, rows, NX, NXp, pitch, r, nshots, scale, g);
        count_launch();
        return cudaGetLastError();
    }
    const long long blocks = std::min<long long>((N + 255) / 256, 152LL * 64);
    probe_dot_kernel<<<(unsigned)blocks, 256, 0, s>>>(Pu, pu_aligned, Pv, N, NX, NXp, pitch, r, nshots, scale, g);
    count_launch();
    return cudaGetLastError();
}

// Row-aligned probe rows (pitch floats, points at row pitch NXp) -> dense layout (N points).
// One warp copies one grid row (NX contiguous floats) of one probe row: no index division
// per element, coalesced on both sides.
__global__ void p_to_user_kernel(const float *__restrict__ in, long long pitch, long long rows, long long N,
                                 int NX, int NXp, long long grows, float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = warp; k < rows * grows; k += nwarps) {
        const long long rw = k / grows, gr = k - rw * grows;
        const float *src = in + rw * pitch + gr * NXp;
        float *dst = out + rw * N + gr * NX;
        for (int x = lane; x < NX; x += 32) dst[x] = src[x];
    }
}

cudaError_t launch_p_to_user(const float *in, long long pitch, long long rows, long long N, int NX,
                             int NXp, float *out, cudaStream_t s)
{
    const long long grows = N / NX;   // (z, y) rows of the grid
    const long long warps = rows * grows;
    const long long blocks = std::min<long long>((warps + 7) / 8, 152LL * 64);
    p_to_user_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, pitch, rows, N, NX, NXp, grows, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
