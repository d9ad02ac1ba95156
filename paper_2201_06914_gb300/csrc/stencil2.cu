// Two time steps per launch of the isotropic acoustic scheme (2-D), the temporal blocking
// of the probed sweeps.
//
// The probed method keeps no wavefield history, so between the two steps of a pair only
// what the probe contraction reads has to reach HBM: the forward increment d^{n+1} (the
// contraction forms u_tt from two increments) or, in the adjoint, v^{j} itself.  u^{n+1}
// stays on chip.  Per shot and point a pair moves 8 B in (u^n, d^n) and 12 B out
// (d^{n+1} or u^{n+1}, then u^{n+2}, d^{n+2}) instead of 32 B for two single steps.
//
// Each step is the arithmetic of stencil_kernel, operation for operation, so a pair gives
// the same bits as two single-step launches.
//
// Tiling.  A block owns TX columns (4 per thread, one float4) and a segment of tz2
// planes.  Stage A computes step 1 on the whole TX-column tile and on the segment
// extended by 4 planes on either side; stage B computes step 2 on the inner TX - 8
// columns (the core) and the segment itself.  Neighbouring tiles overlap by 8 columns and
// neighbouring segments by 8 planes of stage-A work: the halo of step 2 is recomputed
// rather than exchanged.  Stage B trails stage A by 4 planes: u^{n+1} of the own float4
// lives in a register window, its x neighbours in a shared ring of 8 planes, and d^{n+1}
// replaces d^n in the increment ring slot it came from.
//
// Injection uses a CSR table keyed by (tile, plane of the extended segment) that lists
// every entry inside the extended tile (points in an overlap appear in both tiles);
// stage B reads the same keys and keeps the entries of its core.  Each warp sums the
// entries of its own columns in shared memory, so injection needs no block barrier.
//
// Recording: the extra blocks record R u^n from the input and, when the previous launch
// was a pair, the row of its first step as R (u^{n-1} + d^n) from the input of that launch
// and the stored increment, the same addition stage A made.
#include <cstdlib>

#include "stencil_step.cuh"

namespace wp {

using step::P4;


#ifndef WP_STENCIL2_U
#define WP_STENCIL2_U 3
#endif
template <int TXT>
struct Stencil2Shape {
    static constexpr int TX = 4 * TXT;
    static constexpr int C = TX - 2 * RAD;          // core columns (stage B)
    static constexpr int NT = TXT;
    static constexpr int W = TX + 2 * RAD;          // u ring row (x halos of stage A)
    static constexpr int U = WP_STENCIL2_U;         // planes per unrolled group
    static constexpr int LA = 3;                    // planes in flight
    static constexpr int NU = 8;                    // u^n ring: planes z .. z+4+LA
    static constexpr int NDB = 8;                   // d/b ring: planes z-4 .. z+LA
    static constexpr int NV = 8;                    // u^{n+1} ring: planes z-4 .. z
    static constexpr int UCH = W / 4, DBCH = 2 * TX / 4;
    static constexpr int UK = (UCH + NT - 1) / NT, DK = (DBCH + NT - 1) / NT;
    static constexpr size_t SMEM = (size_t)(NU * W + NDB * 2 * TX + NV * TX) * sizeof(float);
    static constexpr int MINB = 8192 / (NT * 24) > 16 ? 16 : 8192 / (NT * 24);
    static_assert(RAD + 1 + LA <= NU && LA + RAD + 1 <= NDB && RAD + 1 <= NV, "rings");
};

template <int TXT, bool WD, bool IMG>
__global__ void __launch_bounds__(TXT, Stencil2Shape<TXT>::MINB) stencil2_kernel(const GridDev G, const StencilArgs A)
{
    using S = Stencil2Shape<TXT>;
    constexpr int TX = S::TX, C = S::C, W = S::W, NT = S::NT, LA = S::LA, U = S::U;
    constexpr int NU = S::NU, NDB = S::NDB, NV = S::NV;
    constexpr uint32_t USZ = W * 4, DSZ = 2 * TX * 4, VSZ = TX * 4;
    extern __shared__ float4 smem4[];
    float *uring = (float *)smem4;
    float *dbring = uring + NU * W;
    float *vring = dbring + NDB * 2 * TX;
    __shared__ float sq[2][TX];   // injected terms [stage][column]
    __shared__ int inj_lo, inj_hi;

    const int ntx = (G.NXp + C - 1) / C;
    const int ntiles = ntx * ((G.NZ + G.tz2 - 1) / G.tz2);
    if ((int)blockIdx.x >= ntiles) {
        gather_rows(A, blockIdx.x - ntiles);
        return;
    }
    const int lx = threadIdx.x, tile = blockIdx.x;
    const long long sh = blockIdx.y;
    const int x0 = (tile % ntx) * C - RAD;
    const int z0 = (tile / ntx) * G.tz2, z1 = min(z0 + G.tz2, G.NZ);
    const int zs = z0 - RAD, ze = z1 + RAD;   // stage-A planes (outside the grid: zeros)
    const int KP = G.tz2 + 2 * RAD;           // table keys per tile
    const int NXp = G.NXp, NZ = G.NZ;
    const float *__restrict__ u = A.u_in + sh * A.u_in_ss;

    uint32_t us[S::UK];
    const float *ug[S::UK];
    int un16[S::UK];
#pragma unroll
    for (int k = 0; k < S::UK; k++) {
        const int c = lx + k * NT;
        const int x = x0 - RAD + 4 * c;
        const bool v = c < S::UCH && x >= 0 && x < NXp;
        un16[k] = v ? 16 : 0;
        us[k] = (uint32_t)(4 * c) * 4;
        ug[k] = u + (v ? x : 0);
    }
    uint32_t ds[S::DK];
    const float *dg[S::DK];
    int dn16[S::DK];
#pragma unroll
    for (int k = 0; k < S::DK; k++) {
        const int c = lx + k * NT;
        const int a = c / (TX / 4), k4 = c % (TX / 4);
        const int x = x0 + 4 * k4;
        const bool v = c < S::DBCH && x >= 0 && x < NXp;
        dn16[k] = v ? 16 : 0;
        ds[k] = (uint32_t)(a * TX + 4 * k4) * 4;
        dg[k] = (a == 1 ? A.b : A.d_in + sh * A.d_in_ss) + (v ? x : 0);
    }
    const uint32_t su0 = (uint32_t)__cvta_generic_to_shared(uring);
    const uint32_t sd0 = (uint32_t)__cvta_generic_to_shared(dbring);
    const uint32_t sv0 = (uint32_t)__cvta_generic_to_shared(vring);
    // plane k of u^n into ring slot (k - zs) mod NU; planes outside the grid are not copied
    // (their slots are never read)
    auto issue_u = [&](int k) {
        if (k < 0 || k >= NZ) return;
        const uint32_t base = su0 + (uint32_t)((k - zs) & (NU - 1)) * USZ;
        const int ko = k * NXp;
#pragma unroll
        for (int q = 0; q < S::UK; q++)
            if ((q + 1) * NT <= S::UCH || lx + q * NT < S::UCH) cp_async16(base + us[q], ug[q] + ko, un16[q]);
    };
    auto issue_db = [&](int k) {
        if (k < 0 || k >= NZ || k >= ze) return;
        const uint32_t base = sd0 + (uint32_t)((k - zs) & (NDB - 1)) * DSZ;
        const int ko = k * NXp;
#pragma unroll
        for (int q = 0; q < S::DK; q++)
            if ((q + 1) * NT <= S::DBCH || lx + q * NT < S::DBCH) cp_async16(base + ds[q], dg[q] + ko, dn16[q]);
    };

#pragma unroll
    for (int k = 0; k < RAD; k++) issue_u(zs + k);
#pragma unroll
    for (int g = 0; g < LA; g++) {
        issue_u(zs + RAD + g);
        issue_db(zs + g);
        cp_async_commit();
    }
    const int *off = A.inj ? A.inj_off + sh * ((long long)ntiles * KP + 1) : nullptr;
    const long long key0 = (long long)tile * KP;
    const bool tile_inj = off && off[key0] < off[key0 + KP];
    if (lx == 0) {
        inj_lo = 1 << 30;
        inj_hi = -1;
    }
    __syncthreads();
    if (tile_inj)
        for (int t = lx; t < KP; t += NT)
            if (off[key0 + t] < off[key0 + t + 1]) {
                atomicMin(&inj_lo, t);
                atomicMax(&inj_hi, t);
            }
    const float *trA = tile_inj ? A.traces + sh * A.tr_ss + (long long)A.step * A.tr_ts : nullptr;
    const float *trB = tile_inj ? A.traces + sh * A.tr_ss + (long long)A.step2 * A.tr_ts : nullptr;

    const int xc = x0 + 4 * lx;
    const bool a_ok = xc >= 0 && xc < NXp;                 // stage-A float4 inside the field
    const bool core = lx >= 1 && lx <= TXT - 2;            // stage-B lanes
    const bool b_ok = a_ok && core;
    float sdx[4];
#pragma unroll
    for (int j = 0; j < 4; j++) sdx[j] = damp_term(xc + j, G.nx, G.nbl, G.hs0x, G.inv_nbl);
    const bool col_int = sdx[0] == 0.f && sdx[1] == 0.f && sdx[2] == 0.f && sdx[3] == 0.f;
    const bool has_pad = xc + 4 > G.NX;
    const long long own = a_ok ? xc : 0;
    float *uo = A.u_out + sh * A.u_out_ss + own;
    float *dout = A.d_out + sh * A.d_out_ss + own;
    float *u1o = A.u1_out ? A.u1_out + sh * A.u1_ss + own : nullptr;
    float *d1o = A.d1_out ? A.d1_out + sh * A.d1_ss + own : nullptr;

    // wa[i]: u^n of plane zb + i - 4; wb[i]: u^{n+1} of plane zb + i - 8 (group start zb)
    P4 wa[2 * RAD + U], wb[2 * RAD + U];
    const P4 zero4 = step::zero();
#pragma unroll
    for (int k = 0; k < RAD; k++) {
        const int zz = zs - RAD + k;
        wa[k] = (a_ok && zz >= 0) ? *(const P4 *)(u + (long long)zz * NXp + own) : zero4;
    }
#pragma unroll
    for (int k = 0; k < 2 * RAD; k++) wb[k] = zero4;
    const uint32_t ub = su0 + (uint32_t)(RAD + 4 * lx) * 4;
    const uint32_t db = sd0 + (uint32_t)(4 * lx) * 4;
    const uint32_t vb = sv0 + (uint32_t)(4 * lx) * 4;
    cp_async_wait<LA - 1>();
    __syncthreads();
    const int klo = inj_lo, khi = inj_hi;
#pragma unroll
    for (int k = 0; k < RAD; k++) {
        const int zz = zs + k;
        wa[RAD + k] = (zz >= 0 && zz < NZ) ? step::lds(ub + (uint32_t)k * USZ) : zero4;
    }

    const int zs0 = G.nbl, zs1 = G.nbl + G.nz;
    const int warp = lx >> 5, lane = lx & 31;
    for (int zb = zs; zb < ze; zb += U) {
#pragma unroll
        for (int ph = 0; ph < U; ph++) {
            const int z = zb + ph;       // stage-A plane
            if (z >= ze) break;
            const int rel = z - zs;
            const int zq = z - RAD;      // stage-B plane
            cp_async_wait<LA - 1>();
            __syncthreads();
            issue_u(z + RAD + LA);
            issue_db(z + LA);
            cp_async_commit();

            wa[2 * RAD + ph] = (z + RAD >= 0 && z + RAD < NZ) ? step::lds(ub + (uint32_t)((rel + RAD) & (NU - 1)) * USZ)
                                                               : zero4;
            const bool actA = z >= 0 && z < NZ;
            const bool actB = zq >= z0 && zq < z1;
            int ea0 = 0, ea1 = 0, eb0 = 0, eb1 = 0;
            if (actA && rel >= klo && rel <= khi) {
                ea0 = off[key0 + rel];
                ea1 = off[key0 + rel + 1];
            }
            if (actB && rel - RAD >= klo && rel - RAD <= khi) {
                eb0 = off[key0 + rel - RAD];
                eb1 = off[key0 + rel - RAD + 1];
            }
            const bool injA = ea1 > ea0, injB = eb1 > eb0;
            if (injA || injB) {
                // each warp sums the entries of its own 128 columns (no block barrier: a
                // lane only reads the float4 of its own columns after the warp's sync)
                *(float4 *)&sq[0][4 * lx] = make_float4(0.f, 0.f, 0.f, 0.f);
                *(float4 *)&sq[1][4 * lx] = make_float4(0.f, 0.f, 0.f, 0.f);
                __syncwarp();
                for (int e = ea0 + lane; e < ea1; e += 32) {
                    const InjEntry E = A.inj[e];
                    if ((E.a >> 7) == warp)
                        atomicAdd(&sq[0][E.a], E.w * A.tr_sign * trA[(long long)E.trace * A.tr_rs]);
                }
                for (int e = eb0 + lane; e < eb1; e += 32) {
                    const InjEntry E = A.inj[e];
                    if ((E.a >> 7) == warp && E.a >= RAD && E.a < TX - RAD)
                        atomicAdd(&sq[1][E.a], E.w * A.tr_sign * trB[(long long)E.trace * A.tr_rs]);
                }
                __syncwarp();
            }

            // ---- stage A: step 1 at plane z on the whole tile
            P4 u1 = zero4;
            float sdv[4];
            if (actA) {
                const uint32_t az = ub + (uint32_t)(rel & (NU - 1)) * USZ;
                const uint32_t adb = db + (uint32_t)(rel & (NDB - 1)) * DSZ;
                const P4 wl = step::lds(az - 16), wr = step::lds(az + 16);
                const P4 din = step::lds(adb), bb = step::lds(adb + TX * 4);
                P4 dn, un;
                step::step4<false, WD>(&wa[ph], nullptr, nullptr, wl, wr, din, bb, &sq[0][4 * lx], injA,
                                   col_int && z >= zs0 && z < zs1, sdx, z, G, dn, un, sdv);
                if (has_pad) step::zero_pad(xc, G.NX, dn, un);
                if (a_ok) {
                    u1 = un;
                    step::sts(adb, dn);   // d^{n+1} replaces d^n: stage B reads it 4 planes later
                    if (core && z >= z0 && z < z1) {
                        const int oz = z * NXp;
                        if (d1o) *(P4 *)(d1o + oz) = dn;
                        if (u1o) *(P4 *)(u1o + oz) = un;
                    }
                }
            }
            step::sts(vb + (uint32_t)(rel & (NV - 1)) * VSZ, u1);
            wb[2 * RAD + ph] = u1;

            // ---- stage B: step 2 at plane z - 4 on the core
            if (actB && b_ok) {
                const int relq = rel - RAD;
                const uint32_t av = vb + (uint32_t)(relq & (NV - 1)) * VSZ;
                const uint32_t adb = db + (uint32_t)(relq & (NDB - 1)) * DSZ;
                const P4 wl = step::lds(av - 16), wr = step::lds(av + 16);
                const P4 din = step::lds(adb), bb = step::lds(adb + TX * 4);
                P4 dn, un;
                step::step4<false, WD>(&wb[ph], nullptr, nullptr, wl, wr, din, bb, &sq[1][4 * lx], injB,
                                   col_int && zq >= zs0 && zq < zs1, sdx, zq, G, dn, un, sdv);
                if (has_pad) step::zero_pad(xc, G.NX, dn, un);
                const int oz = zq * NXp;
                *(P4 *)(uo + oz) = un;
                *(P4 *)(dout + oz) = dn;
                if (IMG) {
                    // exact imaging of both steps at plane zq, one image read and write per
                    // launch: first u_tt of the first step (increments h2, h1) times its
                    // output (the window's centre), then that of the second (h1, h0) times un,
                    // each written as the one-step kernel writes its update, so a pair adds
                    // bit for bit what two single steps add
                    float v1[4], v2[4];
                    step::upk(wb[ph + RAD].a, v1[0], v1[1]);
                    step::upk(wb[ph + RAD].b, v1[2], v1[3]);
                    step::upk(un.a, v2[0], v2[1]);
                    step::upk(un.b, v2[2], v2[3]);
                    const long long p = sh * A.h_ss + oz + own;
                    const float4 h2 = *(const float4 *)(A.h2 + p), h1 = *(const float4 *)(A.h1 + p);
                    const float4 h0 = *(const float4 *)(A.h0 + p);
                    float4 *gi = (float4 *)(A.img + sh * A.img_ss + oz + own);
                    float4 gv = *gi;
                    gv.x += A.img_scale * ((1.f + sdv[0]) * h2.x - (1.f - sdv[0]) * h1.x) * v1[0];
                    gv.y += A.img_scale * ((1.f + sdv[1]) * h2.y - (1.f - sdv[1]) * h1.y) * v1[1];
                    gv.z += A.img_scale * ((1.f + sdv[2]) * h2.z - (1.f - sdv[2]) * h1.z) * v1[2];
                    gv.w += A.img_scale * ((1.f + sdv[3]) * h2.w - (1.f - sdv[3]) * h1.w) * v1[3];
                    gv.x += A.img_scale * ((1.f + sdv[0]) * h1.x - (1.f - sdv[0]) * h0.x) * v2[0];
                    gv.y += A.img_scale * ((1.f + sdv[1]) * h1.y - (1.f - sdv[1]) * h0.y) * v2[1];
                    gv.z += A.img_scale * ((1.f + sdv[2]) * h1.z - (1.f - sdv[2]) * h0.z) * v2[2];
                    gv.w += A.img_scale * ((1.f + sdv[3]) * h1.w - (1.f - sdv[3]) * h0.w) * v2[3];
                    *gi = gv;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 2 * RAD; k++) {
            wa[k] = wa[k + U];
            wb[k] = wb[k + U];
        }
    }
    cp_async_wait<0>();
}

template <int TXT, bool WD, bool IMG = false>
static void launch2_variant(const GridDev &G, const StencilArgs &A, dim3 grid, cudaStream_t s)
{
    using S = Stencil2Shape<TXT>;
    cudaFuncSetAttribute(stencil2_kernel<TXT, WD, IMG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    stencil2_kernel<TXT, WD, IMG><<<grid, S::NT, S::SMEM, s>>>(G, A);
}

template <int TXT>
static void launch2_tiles(const GridDev &G, const StencilArgs &A, cudaStream_t s)
{
    using S = Stencil2Shape<TXT>;
    dim3 grid(stencil2_tiles(G) + gather_blocks(A, S::NT), A.nshots);
    if (A.img) launch2_variant<TXT, false, true>(G, A, grid, s);   // exact adjoint: (u, d) form
    else if (A.wd) launch2_variant<TXT, true>(G, A, grid, s);
    else launch2_variant<TXT, false>(G, A, grid, s);
}

template <int TXT>
static int blocks2_per_sm()
{
    using S = Stencil2Shape<TXT>;
    static int cached = 0;
    if (!cached) {
        cudaFuncSetAttribute(stencil2_kernel<TXT, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stencil2_kernel<TXT, true, false>, S::NT, S::SMEM) != cudaSuccess || n < 1)
            n = 1;
        cached = n;
    }
    return cached;
}

int stencil2_blocks_per_sm(const GridDev &G) { return G.tx == 128 ? blocks2_per_sm<32>() : blocks2_per_sm<64>(); }

cudaError_t launch_stencil2(const GridDev &G, const StencilArgs &A, cudaStream_t s)
{
    if (G.ndim != 2 || G.tti || G.tz2 < 1 || (G.tx != 128 && G.tx != 256)) return cudaErrorInvalidValue;
    if (A.img && A.wd) return cudaErrorInvalidValue;   // the imaging pair is the adjoint's (u, d) form
    const int cls = A.img ? PROF_STENCIL2_IMG : PROF_STENCIL2;
    cudaEvent_t ev = prof_begin(cls, s);
    if (G.tx == 128) launch2_tiles<32>(G, A, s);
    else launch2_tiles<64>(G, A, s);
    prof_end(cls, ev, s);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
