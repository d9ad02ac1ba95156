// Pseudo-acoustic TTI time step (the paper's second physics, Sec. 3 "2007 BP TTI"; the
// paper gives no equations).  Two fields per shot, stored as two consecutive "virtual
// shots" (field p at 2s, field q at 2s+1):
//   m (p_tt + sigma p_t) = E H0 p + S Hz q + src,   m (q_tt + sigma q_t) = S H0 p + Hz q + src
// with E = 1 + 2 eps, S = sqrt(1 + 2 delta), Hz = -Dr^T Dr = sum_i D_i (a_i Dr .),
// Dr = sum_i a_i D_i (8th-order central first derivatives, a = tilted symmetry axis) and
// H0 = L - Hz.  The adjoint applies the transposed block operator: it first combines
// e = E a + S b, f = S a + b and then applies H0 to e and Hz to f.
//
// One step = pass 1 (t_j = Dr x_j for both fields), pass 2 (Hz, L, combination and the
// increment-form leapfrog update of both fields, optionally the exact imaging condition
// summed over both fields), then a point-list injection that adds the linear source term
// to the updated increments and fields.  Both passes are tiled z-marching kernels.
#include <algorithm>

#include "wp_internal.cuh"

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
template <int TX, int TY, bool ADJ>
__global__ void __launch_bounds__(TX *TY) tti_pass1_kernel(const GridDev G, const TtiArgs T, int tz, int ntx,
                                                          int nty)
{
    using S = TtiTile<TX, TY>;
    constexpr int HY = S::HY, WX = S::WX, WY = S::WY, NB = S::NBW;
    __shared__ float s0[WY * WX], s1[WY * WX];
    const int tid = threadIdx.x, lx = tid % TX, ly = tid / TX;
    const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, seg = blockIdx.x / (ntx * nty);
    const long long sh = blockIdx.y;
    const int x0 = bx * TX, y0 = by * TY, z0 = seg * tz, z1 = min(z0 + tz, G.NZ);
    const int x = x0 + lx, y = y0 + ly;
    const long long PS = (long long)G.NXp * G.NY;
    const float *__restrict__ a = T.u_in + (2 * sh) * T.u_in_ss;
    const float *__restrict__ b = T.u_in + (2 * sh + 1) * T.u_in_ss;
    float *t0 = T.t + (2 * sh) * T.t_ss, *t1 = T.t + (2 * sh + 1) * T.t_ss;
    constexpr int NV = ADJ ? 4 : 2;   // raw values per element: a, b (, E, S)
    auto raw = [&](long long q, bool ok, float *v) {
        v[0] = ok ? a[q] : 0.f;
        v[1] = ok ? b[q] : 0.f;
        if (ADJ) {
            v[2] = ok ? T.E[q] : 0.f;
            v[3] = ok ? T.Sd[q] : 0.f;
        }
    };
    auto comb = [&](const float *v, float &x0v, float &x1v) {
        if (ADJ) {
            x0v = v[2] * v[0] + v[3] * v[1];
            x1v = v[3] * v[0] + v[1];
        } else {
            x0v = v[0];
            x1v = v[1];
        }
    };
    Slot sl[NB];
#pragma unroll
    for (int i = 0; i < NB; i++) sl[i] = make_slot(G, tid + i * S::NT, WY * WX, WX, x0 - RAD, y0 - HY);
    const bool own = x < G.NX && y < G.NY;
    const int own_off = own ? y * G.NXp + x : 0;
    const float ihx = 1.f / G.hx, ihy = 1.f / G.hy, ihz = 1.f / G.hz;
    const float cw[4] = {D1C1, D1C2, D1C3, D1C4};
    float w0[2 * RAD + 1], w1[2 * RAD + 1];
#pragma unroll
    for (int k = 0; k < 2 * RAD; k++) {
        const int zz = z0 - RAD + k;
        float v[NV];
        raw((long long)zz * PS + own_off, own && zz >= 0 && zz < G.NZ, v);
        comb(v, w0[k], w1[k]);
    }
    // registers holding the next plane: tile elements and the own column 4 planes ahead
    float tv[NB][NV], ov[NV];
#pragma unroll
    for (int i = 0; i < NB; i++) raw((long long)z0 * PS + sl[i].off, sl[i].ok(), tv[i]);
    raw((long long)(z0 + RAD) * PS + own_off, own && z0 + RAD < G.NZ, ov);
    for (int z = z0; z < z1; z++) {
#pragma unroll
        for (int i = 0; i < NB; i++)
            if (tid + i * S::NT < WY * WX) comb(tv[i], s0[tid + i * S::NT], s1[tid + i * S::NT]);
        comb(ov, w0[2 * RAD], w1[2 * RAD]);
        __syncthreads();
        if (z + 1 < z1) {   // issue the next plane's loads before the arithmetic
#pragma unroll
            for (int i = 0; i < NB; i++) raw((long long)(z + 1) * PS + sl[i].off, sl[i].ok(), tv[i]);
            raw((long long)(z + 1 + RAD) * PS + own_off, own && z + 1 + RAD < G.NZ, ov);
        }
        if (own) {
            float dx0 = 0.f, dx1 = 0.f, dy0 = 0.f, dy1 = 0.f, dz0 = 0.f, dz1 = 0.f;
            const int c0 = (ly + HY) * WX + lx + RAD;
#pragma unroll
            for (int k = 1; k <= RAD; k++) {
                const float c = cw[k - 1];
                dx0 += c * (s0[c0 + k] - s0[c0 - k]);
                dx1 += c * (s1[c0 + k] - s1[c0 - k]);
                if (TY > 1) {
                    dy0 += c * (s0[c0 + k * WX] - s0[c0 - k * WX]);
                    dy1 += c * (s1[c0 + k * WX] - s1[c0 - k * WX]);
                }
                dz0 += c * (w0[RAD + k] - w0[RAD - k]);
                dz1 += c * (w1[RAD + k] - w1[RAD - k]);
            }
            const long long p = (long long)z * PS + own_off;
            const float axv = T.ax[p], azv = T.az[p];
            float acc0 = axv * dx0 * ihx, acc1 = axv * dx1 * ihx;
            if (TY > 1) {
                const float ayv = T.ay[p];
                acc0 += ayv * dy0 * ihy;
                acc1 += ayv * dy1 * ihy;
            }
            t0[p] = acc0 + azv * dz0 * ihz;
            t1[p] = acc1 + azv * dz1 * ihz;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 2 * RAD; k++) {
            w0[k] = w0[k + 1];
            w1[k] = w1[k + 1];
        }
    }
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
    constexpr int NV = ADJ ? 4 : 1;   // raw values of x_0: a (, b, E, S)
    auto raw_x = [&](long long q, bool ok, float *v) {
        v[0] = ok ? a[q] : 0.f;
        if (ADJ) {
            v[1] = ok ? b[q] : 0.f;
            v[2] = ok ? T.E[q] : 0.f;
            v[3] = ok ? T.Sd[q] : 0.f;
        }
    };
    auto x0of = [&](const float *v) { return ADJ ? v[2] * v[0] + v[3] * v[1] : v[0]; };
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
    // registers holding the next plane (raw values; products formed when stored)
    float vx[NXW][3], vy[NYW][3], vb[NB][NV], vo[3 + NV];
    float vc[7];   // own point of the plane: E, S, dt^2/m, both increments, b (and a: zx)
    auto load_plane = [&](int zz) {
        const long long zo = (long long)zz * PS;
        {
            const long long q = zo + own_off;
            vc[0] = own && !ADJ ? T.E[q] : 0.f;
            vc[1] = own && !ADJ ? T.Sd[q] : 0.f;
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
            if (IMG) {
                const float *h1a = T.h1 + (2 * sh) * T.h_ss, *h0a = T.h0 + (2 * sh) * T.h_ss;
                const float *h1b = T.h1 + (2 * sh + 1) * T.h_ss, *h0b = T.h0 + (2 * sh + 1) * T.h_ss;
                const float ua = cp * h1a[p] - cm * h0a[p], ub = cp * h1b[p] - cm * h0b[p];
                T.img[sh * T.img_ss + p] += T.img_scale * (ua * un0 + ub * un1);
            }
        } else if (pad) {
            uo0[p] = uo1[p] = do0[p] = do1[p] = 0.f;
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
    if (T.adjoint) tti_pass1_kernel<TX, TY, true><<<grid, TX * TY, 0, s>>>(G, T, tz, ntx, nty);
    else tti_pass1_kernel<TX, TY, false><<<grid, TX * TY, 0, s>>>(G, T, tz, ntx, nty);
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
