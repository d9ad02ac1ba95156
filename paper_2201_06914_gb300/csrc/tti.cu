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
#include <algorithm>

#include "stencil_step.cuh"

namespace wp {

namespace {

__device__ __forceinline__ void cp_async16(uint32_t dst, const float *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

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

// Both passes march a tile of (x, y) columns along z, one point per thread: in-plane
// neighbours come from shared-memory tiles of the current plane (halo 4, zero outside the
// grid), the 9-plane z neighbourhood of the own column from registers.  Each thread owns
// fixed elements of the tiles (descriptors precomputed once: in-plane offset and whether the
// element lies in the grid) and loads the next plane's elements into registers before it
// computes the current plane, so the load latency overlaps the arithmetic.  Grid:
// blockIdx.x = (x tile, y tile, z segment), blockIdx.y = shot.
template <int TX, int TY>
struct TtiTile {
    static constexpr int HY = TY > 1 ? RAD : 0;
    static constexpr int WX = TX + 2 * RAD;
    static constexpr int WY = TY + 2 * HY;
    static constexpr int NT = TX * TY;
    static constexpr int NXW = (TY * WX + NT - 1) / NT;   // slots of the x-halo tile
    static constexpr int NYW = (WY * TX + NT - 1) / NT;   // slots of the y-halo tile
    static constexpr int NBW = (WY * WX + NT - 1) / NT;   // slots of the both-halo tile
};

// One tile element owned by a thread (element tid + i * NT of the tile): its in-plane
// offset, or -1 when it lies outside the grid in x/y (or beyond the tile).
struct Slot {
    int off;
    __device__ bool ok() const { return off >= 0; }
};

__device__ __forceinline__ Slot make_slot(const GridDev &G, int k, int total, int w, int xs, int ys)
{
    Slot d;
    const int ty = k / w, tx = k - ty * w;
    const int xx = xs + tx, yy = ys + ty;
    const bool ok = k < total && xx >= 0 && xx < G.NX && yy >= 0 && yy < G.NY;
    d.off = ok ? yy * G.NXp + xx : -1;
    return d;
}

// Pass 1: t_j = Dr x_j = sum_i a_i D_i x_j for both fields; x_j are the fields (forward) or
// the combinations e = E a + S b, f = S a + b (adjoint).
//
// Every thread owns two adjacent points of a row (one 8-byte pair) and computes both
// fields with the packed f32x2 instructions.  The x_j tiles of a plane (with x and y
// halos) and the a_x, a_y, a_z tiles of the block's own points are staged by 16-byte
// cp.async copies into a ring of NS planes, LA planes ahead (zero-filled outside the
// grid); the 9-plane z window of the own pair is kept in registers, its newest plane
// loaded from global memory one iteration ahead.
template <int TXP, int TY>
struct Tti1Shape {
    static constexpr int TXT = TXP / 2, NT = TXT * TY;
    static constexpr int HY = TY > 1 ? RAD : 0;
    static constexpr int WX = TXP + 2 * RAD, WY = TY + 2 * HY;
    static constexpr int LA = 2, NS = 4;             // planes in flight; ring slots z .. z+LA
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
__global__ void __launch_bounds__(Tti1Shape<TXP, TY>::NT) tti_pass1_kernel(const GridDev G, const TtiArgs T, int tz,
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
    f2 p0 = ld2(f0, z0 + RAD), p1 = ld2(f1, z0 + RAD);   // the newest window plane, one ahead
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
            p0 = ld2(f0, z + RAD + 1);
            p1 = ld2(f1, z + RAD + 1);
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
template <int TX, int TY, bool ADJ, bool IMG>
__global__ void __launch_bounds__(TX *TY) tti_pass2_kernel(const GridDev G, const TtiArgs T, int tz, int ntx,
                                                          int nty)
{
    using S = TtiTile<TX, TY>;
    constexpr int HY = S::HY, WX = S::WX, WY = S::WY, NXW = S::NXW, NYW = S::NYW, NB = S::NBW;
    __shared__ float wx0[TY * WX], wx1[TY * WX];                                 // a_x t_j, x halo
    __shared__ float wy0[(TY > 1 ? WY : 1) * TX], wy1[(TY > 1 ? WY : 1) * TX];    // a_y t_j, y halo
    __shared__ float sx[WY * WX];                                                // x_0, both halos
    const int tid = threadIdx.x, lx = tid % TX, ly = tid / TX;
    const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, seg = blockIdx.x / (ntx * nty);
    const long long sh = blockIdx.y;
    const int x0 = bx * TX, y0 = by * TY, z0 = seg * tz, z1 = min(z0 + tz, G.NZ);
    const int x = x0 + lx, y = y0 + ly;
    const long long PS = (long long)G.NXp * G.NY;
    const float *__restrict__ a = T.u_in + (2 * sh) * T.u_in_ss;
    const float *__restrict__ b = T.u_in + (2 * sh + 1) * T.u_in_ss;
    const float *__restrict__ t0 = T.t + (2 * sh) * T.t_ss;
    const float *__restrict__ t1 = T.t + (2 * sh + 1) * T.t_ss;
    constexpr int NV = 1;   // x_0: a forward, e adjoint
    const float *__restrict__ x0f = ADJ ? T.ef_in + (2 * sh) * T.ef_ss : a;
    auto raw_x = [&](long long q, bool ok, float *v) { v[0] = ok ? x0f[q] : 0.f; };
    auto x0of = [&](const float *v) { return v[0]; };
    Slot sxs[NXW], sys[NYW], sbs[NB];
#pragma unroll
    for (int i = 0; i < NXW; i++) sxs[i] = make_slot(G, tid + i * S::NT, TY * WX, WX, x0 - RAD, y0);
#pragma unroll
    for (int i = 0; i < NYW; i++) sys[i] = make_slot(G, tid + i * S::NT, WY * TX, TX, x0, y0 - HY);
#pragma unroll
    for (int i = 0; i < NB; i++) sbs[i] = make_slot(G, tid + i * S::NT, WY * WX, WX, x0 - RAD, y0 - HY);
    const bool own = x < G.NX && y < G.NY;
    const bool pad = x >= G.NX && x < G.NXp && y < G.NY;   // row padding: kept at zero
    const int own_off = (own || pad) ? y * G.NXp + x : 0;
    const float ihx = 1.f / G.hx, ihy = 1.f / G.hy, ihz = 1.f / G.hz;
    const float cw[4] = {D1C1, D1C2, D1C3, D1C4};
    const float lw[4] = {WP_C1, WP_C2, WP_C3, WP_C4};
    float zt0[2 * RAD + 1], zt1[2 * RAD + 1], zx[2 * RAD + 1];
    // own column of plane zz: a_z t_0, a_z t_1 and the raw values of x_0
    auto raw_own = [&](int zz, float *v) {
        const bool ok = own && zz >= 0 && zz < G.NZ;
        const long long q = (long long)zz * PS + own_off;
        v[0] = ok ? T.az[q] : 0.f;
        v[1] = ok ? t0[q] : 0.f;
        v[2] = ok ? t1[q] : 0.f;
        raw_x(q, ok, v + 3);
    };
#pragma unroll
    for (int k = 0; k < 2 * RAD; k++) {
        float v[3 + NV];
        raw_own(z0 - RAD + k, v);
        zt0[k] = v[0] * v[1];
        zt1[k] = v[0] * v[2];
        zx[k] = x0of(v + 3);
    }
    float *uo0 = T.u_out + (2 * sh) * T.u_out_ss, *uo1 = T.u_out + (2 * sh + 1) * T.u_out_ss;
    float *do0 = T.d_out + (2 * sh) * T.d_out_ss, *do1 = T.d_out + (2 * sh + 1) * T.d_out_ss;
    const float *di0 = T.d_in + (2 * sh) * T.d_in_ss, *di1 = T.d_in + (2 * sh + 1) * T.d_in_ss;
    float *eo = ADJ ? T.ef_out + (2 * sh) * T.ef_ss : nullptr;
    float *fo = ADJ ? T.ef_out + (2 * sh + 1) * T.ef_ss : nullptr;
    // registers holding the next plane (raw values; products formed when stored)
    float vx[NXW][3], vy[NYW][3], vb[NB][NV], vo[3 + NV];
    float vc[7];   // own point of the plane: E, S, dt^2/m, both increments, b (and a: zx)
    auto load_plane = [&](int zz) {
        const long long zo = (long long)zz * PS;
        {
            const long long q = zo + own_off;
            vc[0] = own ? T.E[q] : 0.f;
            vc[1] = own ? T.Sd[q] : 0.f;
            vc[2] = own ? T.b[q] : 0.f;
            vc[3] = own ? di0[q] : 0.f;
            vc[4] = own ? di1[q] : 0.f;
            vc[5] = own ? b[q] : 0.f;
            vc[6] = own ? a[q] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < NXW; i++) {
            const long long q = zo + sxs[i].off;
            vx[i][0] = sxs[i].ok() ? T.ax[q] : 0.f;
            vx[i][1] = sxs[i].ok() ? t0[q] : 0.f;
            vx[i][2] = sxs[i].ok() ? t1[q] : 0.f;
        }
        if (TY > 1) {
#pragma unroll
            for (int i = 0; i < NYW; i++) {
                const long long q = zo + sys[i].off;
                vy[i][0] = sys[i].ok() ? T.ay[q] : 0.f;
                vy[i][1] = sys[i].ok() ? t0[q] : 0.f;
                vy[i][2] = sys[i].ok() ? t1[q] : 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < NB; i++) raw_x(zo + sbs[i].off, sbs[i].ok(), vb[i]);
        raw_own(zz + RAD, vo);
    };
    load_plane(z0);
    for (int z = z0; z < z1; z++) {
#pragma unroll
        for (int i = 0; i < NXW; i++)
            if (tid + i * S::NT < TY * WX) {
                wx0[tid + i * S::NT] = vx[i][0] * vx[i][1];
                wx1[tid + i * S::NT] = vx[i][0] * vx[i][2];
            }
        if (TY > 1) {
#pragma unroll
            for (int i = 0; i < NYW; i++)
                if (tid + i * S::NT < WY * TX) {
                    wy0[tid + i * S::NT] = vy[i][0] * vy[i][1];
                    wy1[tid + i * S::NT] = vy[i][0] * vy[i][2];
                }
        }
#pragma unroll
        for (int i = 0; i < NB; i++)
            if (tid + i * S::NT < WY * WX) sx[tid + i * S::NT] = x0of(vb[i]);
        zt0[2 * RAD] = vo[0] * vo[1];
        zt1[2 * RAD] = vo[0] * vo[2];
        zx[2 * RAD] = x0of(vo + 3);
        const float cE = vc[0], cS = vc[1], cbm = vc[2], cd0 = vc[3], cd1 = vc[4], cbv = vc[5], cav = vc[6];
        __syncthreads();
        if (z + 1 < z1) load_plane(z + 1);   // next plane's loads overlap this plane's work
        const long long p = (long long)z * PS + own_off;
        if (own) {
            const float c = zx[RAD];
            const int cxw = ly * WX + lx + RAD, cyw = (ly + HY) * TX + lx, cb = (ly + HY) * WX + lx + RAD;
            float hx0 = 0.f, hx1 = 0.f, lx_ = 0.f, hy0 = 0.f, hy1 = 0.f, ly_ = 0.f, hz0 = 0.f, hz1 = 0.f, lz_ = 0.f;
#pragma unroll
            for (int k = 1; k <= RAD; k++) {
                const float cf = cw[k - 1], lf = lw[k - 1];
                hx0 += cf * (wx0[cxw + k] - wx0[cxw - k]);
                hx1 += cf * (wx1[cxw + k] - wx1[cxw - k]);
                lx_ += lf * ((sx[cb + k] + sx[cb - k]) - 2.f * c);
                if (TY > 1) {
                    hy0 += cf * (wy0[cyw + k * TX] - wy0[cyw - k * TX]);
                    hy1 += cf * (wy1[cyw + k * TX] - wy1[cyw - k * TX]);
                    ly_ += lf * ((sx[cb + k * WX] + sx[cb - k * WX]) - 2.f * c);
                }
                hz0 += cf * (zt0[RAD + k] - zt0[RAD - k]);
                hz1 += cf * (zt1[RAD + k] - zt1[RAD - k]);
                lz_ += lf * ((zx[RAD + k] + zx[RAD - k]) - 2.f * c);
            }
            float H0 = hx0 * ihx, H1 = hx1 * ihx, lap = lx_ * G.ihx2;
            if (TY > 1) {
                H0 += hy0 * ihy;
                H1 += hy1 * ihy;
                lap += ly_ * G.ihy2;
            }
            H0 += hz0 * ihz;
            H1 += hz1 * ihz;
            lap += lz_ * G.ihz2;
            float r0, r1;
            if (!ADJ) {
                const float h0p = lap - H0;
                r0 = cE * h0p + cS * H1;
                r1 = cS * h0p + H1;
            } else {
                r0 = lap - H0;
                r1 = H1;
            }
            const float sd = damp_at(G, x, y, z);
            const float cp = 1.f + sd, cm = 1.f - sd;
            const float dn0 = (cm * cd0 + cbm * r0) / cp;
            const float dn1 = (cm * cd1 + cbm * r1) / cp;
            const float un0 = cav + dn0, un1 = cbv + dn1;
            uo0[p] = un0;
            uo1[p] = un1;
            do0[p] = dn0;
            do1[p] = dn1;
            if (ADJ) {
                eo[p] = cE * un0 + cS * un1;
                fo[p] = cS * un0 + un1;
            }
            if (IMG) {
                const float *h1a = T.h1 + (2 * sh) * T.h_ss, *h0a = T.h0 + (2 * sh) * T.h_ss;
                const float *h1b = T.h1 + (2 * sh + 1) * T.h_ss, *h0b = T.h0 + (2 * sh + 1) * T.h_ss;
                const float ua = cp * h1a[p] - cm * h0a[p], ub = cp * h1b[p] - cm * h0b[p];
                T.img[sh * T.img_ss + p] += T.img_scale * (ua * un0 + ub * un1);
            }
        } else if (pad) {
            uo0[p] = uo1[p] = do0[p] = do1[p] = 0.f;
            if (ADJ) eo[p] = fo[p] = 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 2 * RAD; k++) {
            zt0[k] = zt0[k + 1];
            zt1[k] = zt1[k + 1];
            zx[k] = zx[k + 1];
        }
    }
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

template <int TX, int TY>
static void tti_passes(const GridDev &G, const TtiArgs &T, cudaStream_t s)
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
    if (T.img) {
        if (T.adjoint) tti_pass2_kernel<TX, TY, true, true><<<grid, TX * TY, 0, s>>>(G, T, tz, ntx, nty);
        else tti_pass2_kernel<TX, TY, false, true><<<grid, TX * TY, 0, s>>>(G, T, tz, ntx, nty);
    } else {
        if (T.adjoint) tti_pass2_kernel<TX, TY, true, false><<<grid, TX * TY, 0, s>>>(G, T, tz, ntx, nty);
        else tti_pass2_kernel<TX, TY, false, false><<<grid, TX * TY, 0, s>>>(G, T, tz, ntx, nty);
    }
}

cudaError_t launch_tti_step(const GridDev &G, const TtiArgs &T, const TtiInject &J, cudaStream_t s)
{
    cudaEvent_t ev = prof_begin(PROF_STENCIL, s);
    if (G.ndim == 3) tti_passes<32, 8>(G, T, s);
    else tti_passes<128, 1>(G, T, s);
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
