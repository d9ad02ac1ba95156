// Pseudo-acoustic TTI time step (the paper's second physics, Sec. 3 "2007 BP TTI"; the
// paper gives no equations).  Two fields per shot, stored as two consecutive "virtual
// shots" (field p at 2s, field q at 2s+1):
//   m (p_tt + sigma p_t) = E H0 p + S Hz q + src,   m (q_tt + sigma q_t) = S H0 p + Hz q + src
// with E = 1 + 2 eps, S = sqrt(1 + 2 delta), Hz = -Dr^T Dr = sum_i D_i (a_i Dr .),
// Dr = sum_i a_i D_i (8th-order central first derivatives, a = tilted symmetry axis) and
// H0 = L - Hz.  The adjoint applies the transposed block operator: it first combines
// e = E a + S b, f = S a + b and then applies H0 to e and Hz to f.  The adjoint step that
// updates (a, b) also writes the (e, f) of the new fields, so the next step reads them
// directly.
//
// One step = pass 1 (t_j = Dr x_j for both fields), pass 2 (Hz, L, combination and the
// increment-form leapfrog update of both fields, optionally the exact imaging condition
// summed over both fields), then a point-list injection that adds the linear source term
// to the updated increments and fields.  Both passes are tiled z-marching kernels.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "stencil_step.cuh"

namespace wp {

namespace {

constexpr float D1C1 = 4.0f / 5.0f, D1C2 = -1.0f / 5.0f, D1C3 = 4.0f / 105.0f,
                D1C4 = -1.0f / 280.0f;

struct Pt {
    int x, y, z;
};

__device__ __forceinline__ Pt coords(const GridDev &G, long long p)
{
    const long long row = p / G.NXp;
    Pt c;
    c.x = (int)(p - row * G.NXp);
    c.z = (int)(row / G.NY);
    c.y = (int)(row - (long long)c.z * G.NY);
    return c;
}

}  // namespace

// Both passes march a tile of (x, y) points along z (grid: blockIdx.x = (x tile, y tile,
// z segment), blockIdx.y = shot); the in-plane neighbours of a plane come from shared-memory
// tiles with halos of 4 (zero outside the grid), the 9-plane z neighbourhood of a thread's
// own points from registers.

// Pass 1: t_j = Dr x_j = sum_i a_i D_i x_j for both fields; x_j are the fields (forward) or
// the combinations e = E a + S b, f = S a + b (adjoint).
//
// Every thread owns two adjacent points of a row (one 8-byte pair) and computes both
// fields with the packed f32x2 instructions.  The x_j tiles of a plane (with x and y
// halos) and the a_x, a_y, a_z tiles of the block's own points are staged by 16-byte
// cp.async copies into a ring of NS planes, LA planes ahead (zero-filled outside the
// grid); the 9-plane z window of the own pair is kept in registers, its newest plane
// loaded from global memory two iterations ahead.
#ifndef WP_TTI1_LA
#define WP_TTI1_LA 2
#endif
template <int TXP, int TY>
struct Tti1Shape {
    static constexpr int TXT = TXP / 2, NT = TXT * TY;
    static constexpr int HY = TY > 1 ? RAD : 0;
    static constexpr int WX = TXP + 2 * RAD, WY = TY + 2 * HY;
    static constexpr int LA = WP_TTI1_LA, NS = 4;    // planes in flight; ring slots z .. z+LA
    static constexpr int XT = WY * WX;               // floats of one field tile with halos
    static constexpr int AT = TY * TXP;              // floats of one own-point tile
    static constexpr int SLOT = 2 * XT + 3 * AT;     // x_0, x_1; a_x, a_y, a_z
    static constexpr int CH = SLOT / 4;              // 16-byte chunks per slot
    static constexpr int K = (CH + NT - 1) / NT;     // chunks per thread
    static constexpr int U = 2;                      // planes per unrolled group
    static constexpr size_t SMEM = (size_t)NS * SLOT * sizeof(float);
    static_assert(LA + 1 <= NS && (NS & (NS - 1)) == 0, "ring");
    static_assert(TXP % 4 == 0, "tile width");
};

template <int TXP, int TY>
__global__ void __launch_bounds__(Tti1Shape<TXP, TY>::NT, 6) tti_pass1_kernel(const GridDev G, const TtiArgs T, int tz,
                                                                        int ntx, int nty)
{
    using S = Tti1Shape<TXP, TY>;
    using step::f2;
    constexpr int TXT = S::TXT, NT = S::NT, HY = S::HY, WX = S::WX, XT = S::XT, AT = S::AT, LA = S::LA,
                  NS = S::NS, U = S::U;
    constexpr uint32_t SLB = S::SLOT * 4;
    extern __shared__ float4 smem4[];
    const int tid = threadIdx.x, lx = tid % TXT, ly = tid / TXT;
    const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, seg = blockIdx.x / (ntx * nty);
    const long long sh = blockIdx.y;
    const int x0 = bx * TXP, y0 = by * TY, z0 = seg * tz, z1 = min(z0 + tz, G.NZ);
    const int NXp = G.NXp;
    const long long PS = (long long)NXp * G.NY;
    const bool adj = T.adjoint != 0;
    const float *__restrict__ f0 = adj ? T.ef_in + (2 * sh) * T.ef_ss : T.u_in + (2 * sh) * T.u_in_ss;
    const float *__restrict__ f1 = adj ? T.ef_in + (2 * sh + 1) * T.ef_ss : T.u_in + (2 * sh + 1) * T.u_in_ss;
    float *t0 = T.t + (2 * sh) * T.t_ss, *t1 = T.t + (2 * sh + 1) * T.t_ss;

    // copy descriptors (fixed across planes): shared byte offset, source at plane 0, bytes
    uint32_t cd[S::K];
    const float *cs[S::K];
    int cb[S::K];
#pragma unroll
    for (int i = 0; i < S::K; i++) {
        const int c = tid + i * NT;
        int dst = 0, x = -1, y = -1;
        const float *base = f0;
        if (c < 2 * XT / 4) {
            const int f = c / (XT / 4), rem = c % (XT / 4);
            const int r = rem / (WX / 4), k4 = rem % (WX / 4);
            x = x0 - RAD + 4 * k4;
            y = y0 - HY + r;
            dst = f * XT + r * WX + 4 * k4;
            base = f ? f1 : f0;
        } else if (c < S::CH) {
            const int cc = c - 2 * XT / 4;
            const int arr = cc / (AT / 4), rem = cc % (AT / 4);
            const int r = rem / (TXP / 4), k4 = rem % (TXP / 4);
            x = x0 + 4 * k4;
            y = y0 + r;
            dst = 2 * XT + arr * AT + r * TXP + 4 * k4;
            base = arr == 0 ? T.ax : arr == 1 ? T.ay : T.az;
        }
        const bool v = c < S::CH && x >= 0 && x < NXp && y >= 0 && y < G.NY;
        cd[i] = (uint32_t)dst * 4;
        cs[i] = base + (v ? y * NXp + x : 0);
        cb[i] = v ? 16 : 0;
    }
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem4);
    auto issue = [&](int k) {
        if (k >= z1) return;
        const uint32_t base = s0 + (uint32_t)((k - z0) & (NS - 1)) * SLB;
        const long long ko = (long long)k * PS;
#pragma unroll
        for (int i = 0; i < S::K; i++)
            if ((i + 1) * NT <= S::CH || tid + i * NT < S::CH) cp_async16(base + cd[i], cs[i] + ko, cb[i]);
    };
#pragma unroll
    for (int g = 0; g < LA; g++) {
        issue(z0 + g);
        cp_async_commit();
    }

    const int x = x0 + 2 * lx, y = y0 + ly;
    const bool row_ok = x < NXp && y < G.NY;      // the pair lies in the (padded) row
    const long long own = row_ok ? (long long)y * NXp + x : 0;
    auto ld2 = [&](const float *f, int zz) -> f2 {
        return (row_ok && zz >= 0 && zz < G.NZ) ? *(const f2 *)(f + (long long)zz * PS + own) : 0ull;
    };
    f2 w0[2 * RAD + U], w1[2 * RAD + U];   // w[ph + 4 + k]: plane zb + ph + k (group start zb)
#pragma unroll
    for (int k = 0; k < 2 * RAD; k++) {
        w0[k] = ld2(f0, z0 - RAD + k);
        w1[k] = ld2(f1, z0 - RAD + k);
    }
    // the newest window plane (z+4) and the one after it, loaded two iterations ahead
    f2 p0 = ld2(f0, z0 + RAD), p1 = ld2(f1, z0 + RAD);
    f2 n0 = ld2(f0, z0 + RAD + 1), n1 = ld2(f1, z0 + RAD + 1);
    const f2 ihx = step::dup(1.f / G.hx), ihy = step::dup(1.f / G.hy), ihz = step::dup(1.f / G.hz);
    const float cw[4] = {D1C1, D1C2, D1C3, D1C4};
    // pair value lanes: (x + k, x + 1 + k) of a field row from its aligned pairs
    const int cx = (ly + HY) * WX + RAD + 2 * lx;          // float index of x in a field tile
    for (int zb = z0; zb < z1; zb += U) {
#pragma unroll
        for (int ph = 0; ph < U; ph++) {
            const int z = zb + ph;
            if (z >= z1) break;
            cp_async_wait<LA - 1>();
            __syncthreads();
            issue(z + LA);
            cp_async_commit();
            w0[2 * RAD + ph] = p0;
            w1[2 * RAD + ph] = p1;
            p0 = n0;
            p1 = n1;
            n0 = ld2(f0, z + RAD + 2);
            n1 = ld2(f1, z + RAD + 2);
            if (!row_ok) continue;
            const uint32_t sb = s0 + (uint32_t)((z - z0) & (NS - 1)) * SLB;
            f2 t[2];
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const uint32_t fb = sb + (uint32_t)(f * XT + cx) * 4;
                // x neighbours x-4 .. x+5 as five aligned pairs
                f2 q[5];
#pragma unroll
                for (int i = 0; i < 5; i++) q[i] = *(const f2 *)((const char *)smem4 + (fb - s0) + (i - 2) * 8);
                float v[10];
#pragma unroll
                for (int i = 0; i < 5; i++) step::upk(q[i], v[2 * i], v[2 * i + 1]);   // v[j] = x - 4 + j
                f2 dx = 0ull, dy = 0ull, dz = 0ull;
                const f2 *wz = f ? w1 : w0;
#pragma unroll
                for (int k = 1; k <= RAD; k++) {
                    const f2 ck = step::dup(cw[k - 1]);
                    const f2 pp = (k & 1) ? step::pk(v[4 + k], v[5 + k]) : q[2 + k / 2];
                    const f2 pm = (k & 1) ? step::pk(v[4 - k], v[5 - k]) : q[2 - k / 2];
                    dx = step::fma2(ck, step::sub2(pp, pm), dx);
                    if (TY > 1) {
                        const f2 yp = *(const f2 *)((const char *)smem4 + (fb - s0) + k * WX * 4);
                        const f2 ym = *(const f2 *)((const char *)smem4 + (fb - s0) - k * WX * 4);
                        dy = step::fma2(ck, step::sub2(yp, ym), dy);
                    }
                    dz = step::fma2(ck, step::sub2(wz[ph + RAD + k], wz[ph + RAD - k]), dz);
                }
                const char *ab = (const char *)smem4 + (sb - s0) + (2 * XT + ly * TXP + 2 * lx) * 4;
                const f2 axv = *(const f2 *)ab, ayv = *(const f2 *)(ab + AT * 4), azv = *(const f2 *)(ab + 2 * AT * 4);
                f2 acc = step::mul2(step::mul2(axv, dx), ihx);
                if (TY > 1) acc = step::fma2(step::mul2(ayv, dy), ihy, acc);
                t[f] = step::fma2(step::mul2(azv, dz), ihz, acc);
            }
            if (x + 2 > G.NX) {   // row padding: t = 0
                float a0, a1, b0, b1;
                step::upk(t[0], a0, a1);
                step::upk(t[1], b0, b1);
                if (x >= G.NX) a0 = b0 = 0.f;
                a1 = b1 = 0.f;
                t[0] = step::pk(a0, a1);
                t[1] = step::pk(b0, b1);
            }
            const long long p = (long long)z * PS + own;
            *(f2 *)(t0 + p) = t[0];
            *(f2 *)(t1 + p) = t[1];
        }
#pragma unroll
        for (int k = 0; k < 2 * RAD; k++) {
            w0[k] = w0[k + U];
            w1[k] = w1[k + U];
        }
    }
    cp_async_wait<0>();
}

// Pass 2: Hz x_j = sum_i D_i (a_i t_j), L x_0, combination and the increment-form leapfrog
// update of both fields (optionally the exact imaging condition summed over both fields).
//
// Every thread owns two adjacent points of a row and works on pairs with the packed f32x2
// instructions.  One thread of the block stages each plane with tiled TMA copies
// (cp.async.bulk.tensor, zero fill outside the grid) into a ring of NS planes, LA planes
// ahead, completing on the slot's mbarrier: t_0, t_1 and x_0 with x and y halos, a_x with
// the x halo, a_y with the y halo, and the block's own points of E, S, dt^2/m, both
// increments and both fields.  The z neighbourhood of the own pair (a_z t_0, a_z t_1, x_0)
// is a register window whose newest plane is loaded one iteration ahead.
#ifndef WP_TTI2_U
#define WP_TTI2_U 2
#endif
template <int TXP, int TY>
struct Tti2Shape {
    static constexpr int TXT = TXP / 2, NT = TXT * TY;
    static constexpr int HY = TY > 1 ? RAD : 0;
    static constexpr int WX = TXP + 2 * RAD, WY = TY + 2 * HY;
    static constexpr int R32(int n) { return (n + 31) / 32 * 32; }   // 128-byte TMA destinations
    static constexpr int BH = R32(WY * WX), XH = R32(TY * WX), YH = TY > 1 ? R32(WY * TXP) : 0;
    static constexpr int OWN = R32(TY * TXP);
    static constexpr int OT0 = 0, OT1 = BH, OX0 = 2 * BH, OAX = 3 * BH, OAY = OAX + XH, OOWN = OAY + YH;
    static constexpr int NOWN = 7;                   // E, S, dt^2/m, d_0, d_1, a, b
    static constexpr int SLOT = OOWN + NOWN * OWN;   // floats
    static constexpr int LA = 2, NS = 3, U = WP_TTI2_U;
    static constexpr uint32_t TX_BYTES = 4u * (3u * WY * WX + TY * WX + (TY > 1 ? WY * TXP : 0) + NOWN * TY * TXP);
    static constexpr size_t SMEM = (size_t)NS * SLOT * 4 + 128 + 64;
};

// Tensor maps of one pass-2 launch (encoded on the host per launch).
struct Tti2Maps {
    CUtensorMap t;      // [virtual shot][z][y][x] of t, box WX x WY
    CUtensorMap x0;     // x_0 field (a forward, e adjoint), box WX x WY
    CUtensorMap ax;     // [z][y][x], box WX x TY
    CUtensorMap ay;     // box TXP x WY
    CUtensorMap E, S, bm;   // box TXP x TY
    CUtensorMap d;      // increments [virtual shot][z][y][x], box TXP x TY
    CUtensorMap u;      // fields, box TXP x TY
};

__device__ __forceinline__ void tma3(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tma4(void *dst, const CUtensorMap *map, int x, int y, int z, int w, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
                 : "memory");
}

// absorbing-layer term of a pair of points along x (and y); the z term is added per plane
__device__ __forceinline__ step::f2 damp_xy2(const GridDev &G, int x, int y)
{
    const float sy = G.ndim == 3 ? damp_term(y, G.ny, G.nbl, G.hs0y, G.inv_nbl) : 0.f;
    return step::pk(damp_term(x, G.nx, G.nbl, G.hs0x, G.inv_nbl) + sy,
                    damp_term(x + 1, G.nx, G.nbl, G.hs0x, G.inv_nbl) + sy);
}

template <int TXP, int TY, bool ADJ, bool IMG>
__global__ void __launch_bounds__(Tti2Shape<TXP, TY>::NT, 4)
    tti_pass2_kernel(const GridDev G, const TtiArgs T, int tz, int ntx, int nty, const __grid_constant__ Tti2Maps M)
{
    using S = Tti2Shape<TXP, TY>;
    using step::f2;
    using step::pk;
    using step::upk;
    constexpr int TXT = S::TXT, HY = S::HY, WX = S::WX, LA = S::LA, NS = S::NS, U = S::U, OWN = S::OWN;
    extern __shared__ float4 smem4[];
    // 128-byte aligned by pointer arithmetic on the shared array (a shared pointer still)
    float *ring = (float *)((char *)smem4 + ((128u - (smem_u32(smem4) & 127u)) & 127u));
    uint64_t *full = (uint64_t *)(ring + NS * S::SLOT);
    const int tid = threadIdx.x, lx = tid % TXT, ly = tid / TXT;
    const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, seg = blockIdx.x / (ntx * nty);
    const int sh = blockIdx.y;
    const int x0 = bx * TXP, y0 = by * TY, z0 = seg * tz, z1 = min(z0 + tz, G.NZ);
    const int NXp = G.NXp;
    const long long PS = (long long)NXp * G.NY;

    if (tid == 0) {
        for (int i = 0; i < NS; i++) mbar_init(&full[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // producer: all tiles of plane k into ring slot sl
    int nis = 0;   // planes issued (thread 0); slot sl received nis / NS (+1 if sl < nis % NS)
    auto issue = [&](int k, int sl) {
        nis++;
        float *b = ring + sl * S::SLOT;
        uint64_t *bar = &full[sl];
        mbar_arrive_expect_tx(bar, S::TX_BYTES);
        tma4(b + S::OT0, &M.t, x0 - RAD, y0 - HY, k, 2 * sh, bar);
        tma4(b + S::OT1, &M.t, x0 - RAD, y0 - HY, k, 2 * sh + 1, bar);
        tma4(b + S::OX0, &M.x0, x0 - RAD, y0 - HY, k, 2 * sh, bar);
        tma3(b + S::OAX, &M.ax, x0 - RAD, y0, k, bar);
        if (TY > 1) tma3(b + S::OAY, &M.ay, x0, y0 - HY, k, bar);
        float *o = b + S::OOWN;
        tma3(o + 0 * OWN, &M.E, x0, y0, k, bar);
        tma3(o + 1 * OWN, &M.S, x0, y0, k, bar);
        tma3(o + 2 * OWN, &M.bm, x0, y0, k, bar);
        tma4(o + 3 * OWN, &M.d, x0, y0, k, 2 * sh, bar);
        tma4(o + 4 * OWN, &M.d, x0, y0, k, 2 * sh + 1, bar);
        tma4(o + 5 * OWN, &M.u, x0, y0, k, 2 * sh, bar);
        tma4(o + 6 * OWN, &M.u, x0, y0, k, 2 * sh + 1, bar);
    };
    if (tid == 0)
        for (int g = 0; g < LA && z0 + g < z1; g++) issue(z0 + g, g);

    const int x = x0 + 2 * lx, y = y0 + ly;
    const bool row_ok = x < NXp && y < G.NY;
    const bool own = row_ok && x < G.NX;          // first point of the pair inside the row
    const long long own_off = row_ok ? (long long)y * NXp + x : 0;
    const float *__restrict__ t0 = T.t + (2LL * sh) * T.t_ss;
    const float *__restrict__ t1 = T.t + (2LL * sh + 1) * T.t_ss;
    const float *__restrict__ xf = ADJ ? T.ef_in + (2LL * sh) * T.ef_ss : T.u_in + (2LL * sh) * T.u_in_ss;
    auto ld2 = [&](const float *f, int zz) -> f2 {
        return (row_ok && zz >= 0 && zz < G.NZ) ? *(const f2 *)(f + (long long)zz * PS + own_off) : 0ull;
    };
    // z windows: a_z t_0, a_z t_1, x_0 of plane zb + i - 4 at index i (group start zb)
    f2 wa[2 * RAD + U], wb[2 * RAD + U], wx[2 * RAD + U];
#pragma unroll
    for (int k = 0; k < 2 * RAD; k++) {
        const int zz = z0 - RAD + k;
        const f2 az = ld2(T.az, zz);
        wa[k] = step::mul2(az, ld2(t0, zz));
        wb[k] = step::mul2(az, ld2(t1, zz));
        wx[k] = ld2(xf, zz);
    }
    f2 qa = ld2(T.az, z0 + RAD), q0 = ld2(t0, z0 + RAD), q1 = ld2(t1, z0 + RAD), qx = ld2(xf, z0 + RAD);
    float *uo0 = T.u_out + (2LL * sh) * T.u_out_ss, *uo1 = T.u_out + (2LL * sh + 1) * T.u_out_ss;
    float *do0 = T.d_out + (2LL * sh) * T.d_out_ss, *do1 = T.d_out + (2LL * sh + 1) * T.d_out_ss;
    float *eo = ADJ ? T.ef_out + (2LL * sh) * T.ef_ss : nullptr;
    float *fo = ADJ ? T.ef_out + (2LL * sh + 1) * T.ef_ss : nullptr;
    const f2 ihx = step::dup(1.f / G.hx), ihy = step::dup(1.f / G.hy), ihz = step::dup(1.f / G.hz);
    const f2 ihx2 = step::dup(G.ihx2), ihy2 = step::dup(G.ihy2), ihz2 = step::dup(G.ihz2);
    const f2 two = step::dup(2.f), one = step::dup(1.f);
    const float cw[4] = {D1C1, D1C2, D1C3, D1C4};
    const float lw[4] = {WP_C1, WP_C2, WP_C3, WP_C4};
    const int cb = (ly + HY) * WX + RAD + 2 * lx;   // own pair in a both-halo tile
    const int cxh = ly * WX + RAD + 2 * lx;         // own pair in the a_x tile
    const int cyh = (ly + HY) * TXP + 2 * lx;       // own pair in the a_y tile
    const int co = ly * TXP + 2 * lx;               // own pair in an own-point tile
    const f2 sdxy = damp_xy2(G, x, y);
    bool failed = false;
    int sc = 0;                                     // ring slot of plane z
    for (int zb = z0; zb < z1; zb += U) {
#pragma unroll
        for (int ph = 0; ph < U; ph++) {
            const int z = zb + ph;
            if (z >= z1) break;
            if (__syncthreads_or(failed)) goto done;   // slot of plane z-1 is free again
            if (tid == 0 && z + LA < z1) issue(z + LA, sc + LA >= NS ? sc + LA - NS : sc + LA);
            // own pair of plane z+4 enters the windows; plane z+5 is loaded
            wa[2 * RAD + ph] = step::mul2(qa, q0);
            wb[2 * RAD + ph] = step::mul2(qa, q1);
            wx[2 * RAD + ph] = qx;
            qa = ld2(T.az, z + RAD + 1);
            q0 = ld2(t0, z + RAD + 1);
            q1 = ld2(t1, z + RAD + 1);
            qx = ld2(xf, z + RAD + 1);
            const uint32_t parity = (uint32_t)(((z - z0) / NS) & 1);
            if (!mbar_wait_bounded(&full[sc], parity)) {
                failed = true;
                if (T.err) atomicExch(T.err, 1);
            }
            if (!failed && row_ok) {
                const float *sl = ring + sc * S::SLOT;
                const float *o = sl + S::OOWN;
                // x parts: five aligned pairs x-4 .. x+5 of t_0, t_1, x_0 and a_x
                f2 p0[5], p1[5], px[5];
#pragma unroll
                for (int i = 0; i < 5; i++) {
                    const f2 a = *(const f2 *)(sl + S::OAX + cxh + 2 * i - 4);
                    p0[i] = step::mul2(a, *(const f2 *)(sl + S::OT0 + cb + 2 * i - 4));
                    p1[i] = step::mul2(a, *(const f2 *)(sl + S::OT1 + cb + 2 * i - 4));
                    px[i] = *(const f2 *)(sl + S::OX0 + cb + 2 * i - 4);
                }
                auto shifted = [&](const f2 *q, int k) -> f2 {   // (v[x+k], v[x+1+k]), k in -4..4
                    if ((k & 1) == 0) return q[2 + k / 2];
                    float lo0, hi0, lo1, hi1;
                    const int i = (k + 3) >> 1;                 // pair holding x+k as its second lane
                    upk(q[i + 1], lo1, hi1);
                    upk(q[i], lo0, hi0);
                    return pk(hi0, lo1);
                };
                const f2 c = px[2];
                f2 hx0 = 0ull, hx1 = 0ull, lxx = 0ull, hy0 = 0ull, hy1 = 0ull, lyy = 0ull, hz0 = 0ull, hz1 = 0ull, lzz = 0ull;
#pragma unroll
                for (int k = 1; k <= RAD; k++) {
                    const f2 cf = step::dup(cw[k - 1]), lf = step::dup(lw[k - 1]);
                    hx0 = step::fma2(cf, step::sub2(shifted(p0, k), shifted(p0, -k)), hx0);
                    hx1 = step::fma2(cf, step::sub2(shifted(p1, k), shifted(p1, -k)), hx1);
                    lxx = step::fma2(lf, step::sub2(step::add2(shifted(px, k), shifted(px, -k)), step::mul2(two, c)), lxx);
                    if (TY > 1) {
                        const f2 ap = *(const f2 *)(sl + S::OAY + cyh + k * TXP);
                        const f2 am = *(const f2 *)(sl + S::OAY + cyh - k * TXP);
                        const f2 y0p = step::mul2(ap, *(const f2 *)(sl + S::OT0 + cb + k * WX));
                        const f2 y0m = step::mul2(am, *(const f2 *)(sl + S::OT0 + cb - k * WX));
                        const f2 y1p = step::mul2(ap, *(const f2 *)(sl + S::OT1 + cb + k * WX));
                        const f2 y1m = step::mul2(am, *(const f2 *)(sl + S::OT1 + cb - k * WX));
                        hy0 = step::fma2(cf, step::sub2(y0p, y0m), hy0);
                        hy1 = step::fma2(cf, step::sub2(y1p, y1m), hy1);
                        const f2 xp = *(const f2 *)(sl + S::OX0 + cb + k * WX);
                        const f2 xm = *(const f2 *)(sl + S::OX0 + cb - k * WX);
                        lyy = step::fma2(lf, step::sub2(step::add2(xp, xm), step::mul2(two, c)), lyy);
                    }
                    hz0 = step::fma2(cf, step::sub2(wa[ph + RAD + k], wa[ph + RAD - k]), hz0);
                    hz1 = step::fma2(cf, step::sub2(wb[ph + RAD + k], wb[ph + RAD - k]), hz1);
                    lzz = step::fma2(lf, step::sub2(step::add2(wx[ph + RAD + k], wx[ph + RAD - k]), step::mul2(two, c)), lzz);
                }
                f2 H0 = step::mul2(hx0, ihx), H1 = step::mul2(hx1, ihx), lap = step::mul2(lxx, ihx2);
                if (TY > 1) {
                    H0 = step::fma2(hy0, ihy, H0);
                    H1 = step::fma2(hy1, ihy, H1);
                    lap = step::fma2(lyy, ihy2, lap);
                }
                H0 = step::fma2(hz0, ihz, H0);
                H1 = step::fma2(hz1, ihz, H1);
                lap = step::fma2(lzz, ihz2, lap);
                const f2 cE = *(const f2 *)(o + 0 * OWN + co), cS = *(const f2 *)(o + 1 * OWN + co);
                const f2 cbm = *(const f2 *)(o + 2 * OWN + co);
                const f2 cd0 = *(const f2 *)(o + 3 * OWN + co), cd1 = *(const f2 *)(o + 4 * OWN + co);
                const f2 ca = *(const f2 *)(o + 5 * OWN + co), cbv = *(const f2 *)(o + 6 * OWN + co);
                f2 r0, r1;
                if (!ADJ) {
                    const f2 h0p = step::sub2(lap, H0);
                    r0 = step::fma2(cE, h0p, step::mul2(cS, H1));
                    r1 = step::fma2(cS, h0p, H1);
                } else {
                    r0 = step::sub2(lap, H0);
                    r1 = H1;
                }
                const f2 sd = step::add2(sdxy, step::dup(damp_term(z, G.nz, G.nbl, G.hs0z, G.inv_nbl)));
                const f2 cp = step::add2(one, sd), cm = step::sub2(one, sd);
                f2 dn0 = step::fma2(cbm, r0, step::mul2(cm, cd0));
                f2 dn1 = step::fma2(cbm, r1, step::mul2(cm, cd1));
                if (sd != 0ull) {   // inside the absorbing layer: divide by 1 + s
                    float a0, a1, b0, b1, c0, c1;
                    upk(dn0, a0, a1);
                    upk(dn1, b0, b1);
                    upk(cp, c0, c1);
                    dn0 = pk(a0 / c0, a1 / c1);
                    dn1 = pk(b0 / c0, b1 / c1);
                }
                f2 un0 = step::add2(ca, dn0), un1 = step::add2(cbv, dn1);
                f2 e2 = 0ull, f2v = 0ull;
                if (ADJ) {
                    e2 = step::fma2(cE, un0, step::mul2(cS, un1));
                    f2v = step::fma2(cS, un0, un1);
                }
                if (x + 2 > G.NX) {   // row padding: kept at zero
                    auto pad = [&](f2 &v) {
                        float lo, hi;
                        upk(v, lo, hi);
                        v = pk(own ? lo : 0.f, 0.f);
                    };
                    pad(un0);
                    pad(un1);
                    pad(dn0);
                    pad(dn1);
                    pad(e2);
                    pad(f2v);
                }
                const long long p = (long long)z * PS + own_off;
                *(f2 *)(uo0 + p) = un0;
                *(f2 *)(uo1 + p) = un1;
                *(f2 *)(do0 + p) = dn0;
                *(f2 *)(do1 + p) = dn1;
                if (ADJ) {
                    *(f2 *)(eo + p) = e2;
                    *(f2 *)(fo + p) = f2v;
                }
                if (IMG) {
                    const float *h1a = T.h1 + (2LL * sh) * T.h_ss, *h0a = T.h0 + (2LL * sh) * T.h_ss;
                    const float *h1b = T.h1 + (2LL * sh + 1) * T.h_ss, *h0b = T.h0 + (2LL * sh + 1) * T.h_ss;
                    const f2 ua = step::sub2(step::mul2(cp, *(const f2 *)(h1a + p)), step::mul2(cm, *(const f2 *)(h0a + p)));
                    const f2 ub = step::sub2(step::mul2(cp, *(const f2 *)(h1b + p)), step::mul2(cm, *(const f2 *)(h0b + p)));
                    f2 *gi = (f2 *)(T.img + (long long)sh * T.img_ss + p);
                    const f2 add = step::mul2(step::dup(T.img_scale), step::fma2(ua, un0, step::mul2(ub, un1)));
                    f2 g = step::add2(*gi, add);
                    if (x + 2 > G.NX) {
                        float lo, hi;
                        upk(g, lo, hi);
                        g = pk(own ? lo : 0.f, 0.f);
                    }
                    *gi = g;
                }
            }
            sc = sc + 1 == NS ? 0 : sc + 1;
        }
#pragma unroll
        for (int k = 0; k < 2 * RAD; k++) {
            wa[k] = wa[k + U];
            wb[k] = wb[k + U];
            wx[k] = wx[k + U];
        }
    }
done:
    // after a failed wait, let the copies in flight land before the block's memory is reused
    if (__syncthreads_or(failed) && tid == 0)
        for (int i = 0; i < NS; i++) {
            const int cnt = nis / NS + (i < nis % NS ? 1 : 0);
            if (cnt > 0) (void)mbar_wait_bounded(&full[i], (uint32_t)((cnt - 1) & 1));
        }
    __syncthreads();
}

// Adds the source term after the update: a point source value q at point p changes the
// increment and the field by (dt^2/m) q / (1 + sigma dt/2) (the update is linear in q).
// Forward: both fields; adjoint: the p-equation only.  The exact imaging condition gets
// the matching correction.
__global__ void tti_inject_kernel(const GridDev G, const TtiArgs T, const int *idx, const float *w,
                                  int npts, int ncorner, const float *traces, long long tr_ss,
                                  long long tr_ts, long long tr_rs, int step, float sign, int both)
{
    const long long sh = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npts * ncorner) return;
    const int j = e / ncorner;
    const long long k = ((long long)sh * npts + j) * ncorner + (e % ncorner);
    const long long p = idx[k];
    const float val = sign * w[k] * traces[sh * tr_ss + (long long)step * tr_ts + j * tr_rs];
    const Pt c = coords(G, p);
    const float sd = damp_at(G, c.x, c.y, c.z);
    const float dd = T.b[p] * val / (1.f + sd);
    for (int f = 0; f < (both ? 2 : 1); f++) {
        atomicAdd(T.d_out + (2 * sh + f) * T.d_out_ss + p, dd);
        atomicAdd(T.u_out + (2 * sh + f) * T.u_out_ss + p, dd);
    }
    if (T.adjoint) {   // the p-field change enters e = E a + S b and f = S a + b
        atomicAdd(T.ef_out + (2 * sh) * T.ef_ss + p, T.E[p] * dd);
        atomicAdd(T.ef_out + (2 * sh + 1) * T.ef_ss + p, T.Sd[p] * dd);
    }
    if (T.img) {
        const float ua = (1.f + sd) * T.h1[(2 * sh) * T.h_ss + p] - (1.f - sd) * T.h0[(2 * sh) * T.h_ss + p];
        atomicAdd(T.img + sh * T.img_ss + p, T.img_scale * ua * dd);
    }
}

// E, S and the tilted axis (ax, ay, az) on the padded layout from the user-layout fields.
__global__ void tti_params_kernel(const GridDev G, const float *eps, const float *delta,
                                  const float *theta, const float *phi, float *E, float *Sd,
                                  float *ax, float *ay, float *az)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < G.Np;
         p += (long long)gridDim.x * blockDim.x) {
        const long long row = p / G.NXp;
        const int x = (int)(p - row * G.NXp);
        if (x >= G.NX) {
            E[p] = Sd[p] = ax[p] = ay[p] = az[p] = 0.f;
            continue;
        }
        const long long u = row * G.NX + x;
        const float th = theta[u], ph = (G.ndim == 3 && phi) ? phi[u] : 0.f;
        E[p] = 1.f + 2.f * eps[u];
        Sd[p] = sqrtf(1.f + 2.f * delta[u]);
        ax[p] = sinf(th) * cosf(ph);
        ay[p] = sinf(th) * sinf(ph);
        az[p] = cosf(th);
    }
}

static unsigned blocks_for(long long n)
{
    const long long g = (n + 255) / 256;
    return (unsigned)(g < 152LL * 32 ? g : 152LL * 32);
}

cudaError_t launch_tti_params(const GridDev &G, const float *eps, const float *delta,
                              const float *theta, const float *phi, float *E, float *Sd,
                              float *ax, float *ay, float *az, cudaStream_t s)
{
    tti_params_kernel<<<blocks_for(G.Np), 256, 0, s>>>(G, eps, delta, theta, phi, E, Sd, ax, ay, az);
    count_launch();
    return cudaGetLastError();
}

typedef CUresult (*tti_encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static tti_encode_fn tti_encoder()
{
    static tti_encode_fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (tti_encode_fn)p;
    }
    return fn;
}

// A tiled float map over [w][z][y][x] (rank 4, w_ss floats between w slices) or [z][y][x]
// (rank 3) of a padded field; out-of-range elements read as zero.
static bool tti_map(CUtensorMap *m, const float *base, const GridDev &G, int rank, long long nw, long long w_ss,
                    uint32_t bx, uint32_t by)
{
    tti_encode_fn enc = tti_encoder();
    if (!enc || ((uintptr_t)base & 15) || (w_ss & 3)) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)G.NXp, (cuuint64_t)G.NY, (cuuint64_t)G.NZ, (cuuint64_t)nw};
    const cuuint64_t strides[3] = {(cuuint64_t)G.NXp * 4, (cuuint64_t)G.NXp * G.NY * 4, (cuuint64_t)w_ss * 4};
    const cuuint32_t box[4] = {bx, by, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, (void *)base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int TX, int TY>
static cudaError_t tti_passes(const GridDev &G, const TtiArgs &T, cudaStream_t s)
{
    const int ntx = (G.NX + TX - 1) / TX, nty = (G.NY + TY - 1) / TY;
    // z segments: about four waves of 8 resident blocks per SM, marches of >= 16 planes
    const long long cols = (long long)ntx * nty * T.nshots;
    const long long want = 4LL * device_sm_count() * 8;
    int nseg = (int)std::max<long long>(1, (want + cols - 1) / cols);
    int tz = (G.NZ + nseg - 1) / nseg;
    tz = std::max(tz, std::min(16, G.NZ));
    nseg = (G.NZ + tz - 1) / tz;
    dim3 grid((unsigned)((long long)ntx * nty * nseg), T.nshots);
    using S1 = Tti1Shape<TX, TY>;
    cudaFuncSetAttribute(tti_pass1_kernel<TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S1::SMEM);
    tti_pass1_kernel<TX, TY><<<grid, S1::NT, S1::SMEM, s>>>(G, T, tz, ntx, nty);

    using S2 = Tti2Shape<TX, TY>;
    Tti2Maps M;
    memset(&M, 0, sizeof M);
    const long long nv = 2LL * T.nshots;
    const float *xf = T.adjoint ? T.ef_in : T.u_in;
    const long long xss = T.adjoint ? T.ef_ss : T.u_in_ss;
    bool ok = tti_map(&M.t, T.t, G, 4, nv, T.t_ss, S2::WX, S2::WY) &&
              tti_map(&M.x0, xf, G, 4, nv, xss, S2::WX, S2::WY) &&
              tti_map(&M.ax, T.ax, G, 3, 1, 0, S2::WX, TY) &&
              tti_map(&M.ay, T.ay, G, 3, 1, 0, TX, S2::WY) &&
              tti_map(&M.E, T.E, G, 3, 1, 0, TX, TY) && tti_map(&M.S, T.Sd, G, 3, 1, 0, TX, TY) &&
              tti_map(&M.bm, T.b, G, 3, 1, 0, TX, TY) &&
              tti_map(&M.d, T.d_in, G, 4, nv, T.d_in_ss, TX, TY) &&
              tti_map(&M.u, T.u_in, G, 4, nv, T.u_in_ss, TX, TY);
    if (!ok) return cudaErrorInvalidValue;
    auto run = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S2::SMEM);
        kern<<<grid, S2::NT, S2::SMEM, s>>>(G, T, tz, ntx, nty, M);
    };
    if (T.img) {
        if (T.adjoint) run(tti_pass2_kernel<TX, TY, true, true>);
        else run(tti_pass2_kernel<TX, TY, false, true>);
    } else {
        if (T.adjoint) run(tti_pass2_kernel<TX, TY, true, false>);
        else run(tti_pass2_kernel<TX, TY, false, false>);
    }
    return cudaSuccess;
}

cudaError_t launch_tti_step(const GridDev &G, const TtiArgs &T, const TtiInject &J, cudaStream_t s)
{
    cudaEvent_t ev = prof_begin(PROF_STENCIL, s);
    const cudaError_t e = G.ndim == 3 ? tti_passes<32, 8>(G, T, s) : tti_passes<128, 1>(G, T, s);
    if (e != cudaSuccess) return e;
    count_launch(2);
    if (J.npts > 0) {
        dim3 g2((J.npts * J.ncorner + 255) / 256, T.nshots);
        tti_inject_kernel<<<g2, 256, 0, s>>>(G, T, J.idx, J.w, J.npts, J.ncorner, J.traces, J.tr_ss,
                                             J.tr_ts, J.tr_rs, J.step, J.sign, J.both);
        count_launch();
    }
    prof_end(PROF_STENCIL, ev, s);
    return cudaGetLastError();
}

}  // namespace wp
