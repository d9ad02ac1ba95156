// Pipelined probe accumulation on the tensor cores (Eq. 3), the hot-path version of
// probe_gemm.cu.  For every shot and every 128-point tile of the grid:
//   P[i][x] += scale * sum_{t < cnt} A[t][x] * Q[t0 + t][i]
// where A is read from the time-step ring (forward: u_tt rebuilt from two consecutive
// stored increments; adjoint: the adjoint wavefield itself).
//
// One persistent CTA per SM runs a warp-specialised pipeline over its (shot, tile) items:
//   warp 8     producer: per 64-step chunk, 64 (or 65) bulk copies of 512-byte ring rows
//              plus two pre-swizzled probe images (bf16 hi/lo) into a stage of shared
//              memory, completing on the stage's `full` mbarrier;
//   warps 0-3  converters: one grid point per thread, FP32 -> u_tt (or v) -> bfloat16
//              hi + lo, written in the K-major 128-byte-swizzled layout tcgen05 reads;
//   warp 9     MMA issuer (one thread): 4 bf16 products per 16-step k-slice into a
//              double-buffered TMEM accumulator; commits release the stage and, after the
//              last chunk of an item, hand the accumulator to the epilogue;
//   warps 4-7  epilogue: tcgen05.ld of the accumulator, read-modify-write of P in global
//              memory (and, after the last adjoint block, the randomized imaging condition).
// Every wait is bounded; a wait that gives up raises the kernel error flag and all roles
// leave their loops, the TMEM is freed and the kernel returns.
#include <algorithm>

#include "wp_internal.cuh"

namespace wp {

namespace {

constexpr int PIPE_THREADS = 320;
constexpr int CH = 64;                    // time steps per chunk
constexpr uint32_t A32_BYTES = 33792;     // 65 rows x 512 B, rounded to 1 KiB

__host__ __device__ inline uint32_t pipe_cols(int r_pad)
{
    uint32_t c = 32;
    while (c < (uint32_t)r_pad) c <<= 1;
    return c;
}

// Stage = [A region: 65 FP32 ring rows, overwritten in place by the bf16 hi/lo operand
//          (2 x 16 KiB) once all converter threads have read their column]
//         [probe image hi][probe image lo]
__host__ __device__ inline uint32_t stage_bytes(int r_pad)
{
    return A32_BYTES + 2u * (uint32_t)r_pad * 128u;
}

// Named barrier over the 128 converter threads that also returns, to every one of them,
// whether any of them failed its wait: the converters leave their loops together, so no
// thread is left waiting at the barrier for one that has gone.
__device__ __forceinline__ bool converters_any(bool failed)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred q, p;\n\t"
                 "setp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.or.pred p, 1, 128, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r) : "r"((uint32_t)failed) : "memory");
    return r != 0;
}

__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > (1ll << 31)) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ uint32_t pack2(float a, float b, bool lo_part)
{
    const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    if (!lo_part)
        return (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
    const __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
    const __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
    return (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
}

}  // namespace

__global__ void __launch_bounds__(PIPE_THREADS, 1) probe_pipe_kernel(const PipeArgs A, int ST, int nshots)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[4], empty[4], aready[4], accfull[2], accempty[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t SB = stage_bytes(A.r_pad);
    const uint32_t ncols = pipe_cols(A.r_pad);
    const int nitems = A.ntiles * nshots;
    const int nch = (A.cnt + CH - 1) / CH;

    if (tid == 0) {
        for (int s = 0; s < ST; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            mbar_init(&aready[s], 128);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], 128);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 9) tmem_alloc(&tmem_holder, 2 * ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;

    auto stage_ptr = [&](int s) { return smem + (size_t)s * SB; };

    if (warp == 8) {
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
                if (lane == 0) mbar_arrive_expect_tx(&full[s], (uint32_t)(rows * 512 + 2 * img_bytes));
                __syncwarp();
                for (int t = lane; t < rows; t += 32) {
                    const int slot = (A.slot0 + c * CH + t) % A.nslots;
                    bulk_g2s(st + (size_t)t * 512, ring + (long long)slot * A.sstride, 512, &full[s]);
                }
                if (lane == 0) {
                    const long long im = ((long long)(shot / A.img_div) * A.nblocks + A.blk) * A.ncb + c;
                    const uint8_t *hi = (const uint8_t *)A.img_hi + im * img_bytes;
                    const uint8_t *lo = (const uint8_t *)A.img_lo + im * img_bytes;
                    bulk_g2s(st + A32_BYTES, hi, (uint32_t)img_bytes, &full[s]);
                    bulk_g2s(st + A32_BYTES + img_bytes, lo, (uint32_t)img_bytes, &full[s]);
                }
                __syncwarp();
            }
        }
    } else if (warp == 9) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(128, A.r_pad);
            const uint32_t img_bytes = (uint32_t)A.r_pad * 128;
            uint32_t g = 0, j = 0;
            for (int item = blockIdx.x; item < nitems && !abort_flag; item += gridDim.x, j++) {
                const int ab = j & 1;
                if (!wait_bar(&accempty[ab], ((j >> 1) & 1) ^ 1, &abort_flag)) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)ab * ncols;
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
                        umma_bf16(dt, dah, dbh, idesc, (c > 0 || k > 0) ? 1u : 0u);
                        umma_bf16(dt, dal, dbh, idesc, 1u);
                        umma_bf16(dt, dah, dbl, idesc, 1u);
                        umma_bf16(dt, dal, dbl, idesc, 1u);
                    }
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&accfull[ab]);
            }
        }
    } else if (warp < 4) {
        // ---------------- converters ----------------
        const int m = tid;
        uint32_t g = 0;
        // No early exit on the abort flag here: a failed wait is voted on by all converters
        for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
            const int tile = item % A.ntiles;
            const long long p = (long long)tile * 128 + m;
            const long long prow = p / A.NXp;
            const bool valid = p < A.Np && (int)(p - prow * A.NXp) < A.NX;
            float cp = 1.f, cm = 1.f;
            if (A.mode == 1 && valid) {
                const int x = (int)(p - prow * A.NXp);
                const int z = (int)(prow / A.G.NY), y = (int)(prow - (long long)z * A.G.NY);
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
                const int need = A.cnt - c * CH;
                const bool rd = valid && got;
                float v[CH];
                if (A.mode == 0) {
#pragma unroll
                    for (int t = 0; t < CH; t++) v[t] = (rd && t < need) ? a32[t * 128 + m] : 0.f;
                } else {
                    float prev = rd ? a32[m] : 0.f;
#pragma unroll
                    for (int t = 0; t < CH; t++) {
                        const bool in = rd && t < need;
                        const float nx = in ? a32[(t + 1) * 128 + m] : 0.f;
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
                for (int cc = 0; cc < 8; cc++) {
                    const uint32_t off = (uint32_t)m * 128u + ((uint32_t)(cc ^ (m & 7)) << 4);
                    const float *x = v + cc * 8;
                    *(uint4 *)(ah + off) = make_uint4(pack2(x[0], x[1], false), pack2(x[2], x[3], false),
                                                      pack2(x[4], x[5], false), pack2(x[6], x[7], false));
                    *(uint4 *)(al + off) = make_uint4(pack2(x[0], x[1], true), pack2(x[2], x[3], true),
                                                      pack2(x[4], x[5], true), pack2(x[6], x[7], true));
                }
                fence_proxy_async_smem();
                mbar_arrive(&aready[s]);
            }
            if (!ok) break;
        }
    } else {
        // ---------------- epilogue (warps 4-7) ----------------
        // The old values of the first 64 probe columns of the next item are loaded while
        // that item's MMAs run, so the read-modify-write of P costs no exposed latency.
        constexpr int PF = 64;
        const int e = tid - 128, ew = warp - 4;
        float pre[PF];
        // ring point p (pitch NXp) -> user point (pitch NX), or -1 for padding
        auto user_index = [&](int tile) -> long long {
            const long long p = (long long)tile * 128 + e;
            const long long prow = p / A.NXp;
            const int x = (int)(p - prow * A.NXp);
            return (p < A.Np && x < A.NX) ? prow * A.NX + x : -1;
        };
        auto prefetch = [&](int item) {
            const int shot = item / A.ntiles, tile = item % A.ntiles;
            const long long pu = user_index(tile);
            const float *P = A.P + (long long)shot * A.P_ss + (pu < 0 ? 0 : pu);
#pragma unroll
            for (int q = 0; q < PF; q++)
                pre[q] = (!A.p_zero && pu >= 0 && q < A.r) ? P[(long long)q * A.N] : 0.f;
        };
        if ((int)blockIdx.x < nitems) prefetch(blockIdx.x);
        uint32_t j = 0;
        for (int item = blockIdx.x; item < nitems && !abort_flag; item += gridDim.x, j++) {
            const int shot = item / A.ntiles, tile = item % A.ntiles;
            const int ab = j & 1;
            if (!wait_bar(&accfull[ab], (j >> 1) & 1, &abort_flag)) break;
            tc_fence_after();
            const long long pu = user_index(tile);
            const bool valid = pu >= 0;
            const long long p = valid ? pu : 0;
            float *P = A.P + (long long)shot * A.P_ss + p;
            const float *Pu = A.do_img ? A.Pu + (long long)shot * A.Pu_ss + p : nullptr;
            float img = 0.f;
            const uint32_t taddr = tmem + (uint32_t)ab * ncols + ((uint32_t)(ew * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < PF; c0 += 16) {
                if (c0 < A.r_pad) {
                    uint32_t r16[16];
                    tmem_ld16(taddr + (uint32_t)c0, r16);
#pragma unroll
                    for (int q = 0; q < 16; q++) {
                        const int i = c0 + q;
                        if (valid && i < A.r) {
                            const float nv = pre[i] + A.scale * __uint_as_float(r16[q]);
                            P[(long long)i * A.N] = nv;
                            if (Pu) img += Pu[(long long)i * A.N] * nv;
                        }
                    }
                }
            }
            for (int c0 = PF; c0 < A.r_pad; c0 += 16) {
                uint32_t r16[16];
                tmem_ld16(taddr + (uint32_t)c0, r16);
                if (valid) {
                    float old[16];
#pragma unroll
                    for (int q = 0; q < 16; q++)
                        old[q] = (!A.p_zero && c0 + q < A.r) ? P[(long long)(c0 + q) * A.N] : 0.f;
#pragma unroll
                    for (int q = 0; q < 16; q++) {
                        if (c0 + q < A.r) {
                            const float nv = old[q] + A.scale * __uint_as_float(r16[q]);
                            P[(long long)(c0 + q) * A.N] = nv;
                            if (Pu) img += Pu[(long long)(c0 + q) * A.N] * nv;
                        }
                    }
                }
            }
            if (Pu && valid) A.img[(long long)shot * A.img_ss + p] = A.img_scale * img;
            tc_fence_before();
            mbar_arrive(&accempty[ab]);
            if (item + (int)gridDim.x < nitems) prefetch(item + gridDim.x);
        }
    }

    __syncthreads();
    if (abort_flag && tid == 0) atomicExch(A.err, 2);
    if (warp == 9) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * ncols);
    }
}

static int g_num_sms = 0;

cudaError_t launch_probe_pipe(const PipeArgs &A, int nshots, cudaStream_t s)
{
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    const uint32_t SB = stage_bytes(A.r_pad);
    const size_t avail = 227 * 1024 - 1024 - 256;
    int ST = (int)std::min<size_t>(4, avail / SB);
    if (ST < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)ST * SB + 1024;
    cudaError_t e = cudaFuncSetAttribute(probe_pipe_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long items = (long long)A.ntiles * nshots;
    if (items >= (1LL << 31)) return cudaErrorInvalidValue;
    dim3 grid((unsigned)std::min<long long>(items, g_num_sms));
    cudaEvent_t ev = prof_begin(PROF_GEMM, s);
    probe_pipe_kernel<<<grid, PIPE_THREADS, smem, s>>>(A, ST, nshots);
    prof_end(PROF_GEMM, ev, s);
    count_launch();
    return cudaGetLastError();
}

// Swizzled probe images.  Image (shot, b, c) holds rows i < r_pad and 64 columns k, value
// Q[shot][t][i] for t = t_first + b*Tb + c*64 + k inside block b and below nt (else 0),
// split into bf16 hi and lo; byte offset of (i, k): i*128 + (((k/8) ^ (i%8)) * 16) + (k%8)*2.
__global__ void probe_image_kernel(const float *Q, int nt, int r, int r_pad, int t_first, int Tb,
                                   int nblocks, int ncb, __nv_bfloat16 *hi, __nv_bfloat16 *lo)
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
}

cudaError_t launch_probe_images(const float *Q, int nshots, int nt, int r, int r_pad,
                                int t_first, int Tb, int nblocks, __nv_bfloat16 *hi,
                                __nv_bfloat16 *lo, cudaStream_t s)
{
    const int ncb = (Tb + 63) / 64;
    dim3 grid((unsigned)((long long)nshots * nblocks * ncb), r_pad);
    probe_image_kernel<<<grid, 64, 0, s>>>(Q, nt, r, r_pad, t_first, Tb, nblocks, ncb, hi, lo);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
