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
// grid), the 9-plane z neighbourhood of the own column from registers.  Grid: blockIdx.x =
// (x tile, y tile, z segment), blockIdx.y = shot.
template <int TX, int TY>
struct TtiTile {
    static constexpr int HY = TY > 1 ? RAD : 0;
    static constexpr int WX = TX + 2 * RAD;
    static constexpr int WY = TY + 2 * HY;
    static constexpr int NT = TX * TY;
};

__device__ __forceinline__ bool in_grid(const GridDev &G, int x, int y, int z)
{
    return x >= 0 && x < G.NX && y >= 0 && y < G.NY && z >= 0 && z < G.NZ;
}

// Pass 1: t_j = Dr x_j = sum_i a_i D_i x_j for both fields; x_j are the fields (forward) or
// the combinations e = E a + S b, f = S a + b (adjoint).
template <int TX, int TY, bool ADJ>
__global__ void __launch_bounds__(TX *TY) tti_pass1_kernel(const GridDev G, const TtiArgs T, int tz, int ntx,
                                                          int nty)
{
    using S = TtiTile<TX, TY>;
    constexpr int HY = S::HY, WX = S::WX, WY = S::WY;
    __shared__ float s0[WY][WX], s1[WY][WX];
    const int tid = threadIdx.x, lx = tid % TX, ly = tid / TX;
    const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, seg = blockIdx.x / (ntx * nty);
    const long long sh = blockIdx.y;
    const int x0 = bx * TX, y0 = by * TY, z0 = seg * tz, z1 = min(z0 + tz, G.NZ);
    const int x = x0 + lx, y = y0 + ly;
    const long long PS = (long long)G.NXp * G.NY;
    const float *__restrict__ a = T.u_in + (2 * sh) * T.u_in_ss;
    const float *__restrict__ b = T.u_in + (2 * sh + 1) * T.u_in_ss;
    float *t0 = T.t + (2 * sh) * T.t_ss, *t1 = T.t + (2 * sh + 1) * T.t_ss;
    auto val = [&](int xx, int yy, int zz, float &v0, float &v1) {
        if (!in_grid(G, xx, yy, zz)) {
            v0 = v1 = 0.f;
            return;
        }
        const long long q = (long long)zz * PS + (long long)yy * G.NXp + xx;
        const float av = a[q], bv = b[q];
        if (ADJ) {
            const float e = T.E[q], sd = T.Sd[q];
            v0 = e * av + sd * bv;
            v1 = sd * av + bv;
        } else {
            v0 = av;
            v1 = bv;
        }
    };
    const bool own = x < G.NX && y < G.NY;
    const float ihx = 1.f / G.hx, ihy = 1.f / G.hy, ihz = 1.f / G.hz;
    const float cw[4] = {D1C1, D1C2, D1C3, D1C4};
    float w0[2 * RAD + 1], w1[2 * RAD + 1];
#pragma unroll
    for (int k = 0; k < 2 * RAD; k++) val(x, y, z0 - RAD + k, w0[k], w1[k]);
    for (int z = z0; z < z1; z++) {
        val(x, y, z + RAD, w0[2 * RAD], w1[2 * RAD]);
        for (int k = tid; k < WX * WY; k += S::NT) {
            const int ty = k / WX, tx = k - ty * WX;
            val(x0 - RAD + tx, y0 - HY + ty, z, s0[ty][tx], s1[ty][tx]);
        }
        __syncthreads();
        if (own) {
            float dx0 = 0.f, dx1 = 0.f, dy0 = 0.f, dy1 = 0.f, dz0 = 0.f, dz1 = 0.f;
#pragma unroll
            for (int k = 1; k <= RAD; k++) {
                const float c = cw[k - 1];
                dx0 += c * (s0[ly + HY][lx + RAD + k] - s0[ly + HY][lx + RAD - k]);
                dx1 += c * (s1[ly + HY][lx + RAD + k] - s1[ly + HY][lx + RAD - k]);
                if (TY > 1) {
                    dy0 += c * (s0[ly + HY + k][lx + RAD] - s0[ly + HY - k][lx + RAD]);
                    dy1 += c * (s1[ly + HY + k][lx + RAD] - s1[ly + HY - k][lx + RAD]);
                }
                dz0 += c * (w0[RAD + k] - w0[RAD - k]);
                dz1 += c * (w1[RAD + k] - w1[RAD - k]);
            }
            const long long p = (long long)z * PS + (long long)y * G.NXp + x;
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
    constexpr int HY = S::HY, WX = S::WX, WY = S::WY;
    __shared__ float wx0[TY][WX], wx1[TY][WX];                                  // a_x t_j, x halo
    __shared__ float wy0[TY > 1 ? WY : 1][TX], wy1[TY > 1 ? WY : 1][TX];          // a_y t_j, y halo
    __shared__ float sx[WY][WX];                                                 // x_0, both halos
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
    auto qof = [&](int xx, int yy, int zz) { return (long long)zz * PS + (long long)yy * G.NXp + xx; };
    auto x0val = [&](long long q) { return ADJ ? T.E[q] * a[q] + T.Sd[q] * b[q] : a[q]; };
    const bool own = x < G.NX && y < G.NY;
    const bool pad = x >= G.NX && x < G.NXp && y < G.NY;   // row padding: kept at zero
    const float ihx = 1.f / G.hx, ihy = 1.f / G.hy, ihz = 1.f / G.hz;
    const float cw[4] = {D1C1, D1C2, D1C3, D1C4};
    const float lw[4] = {WP_C1, WP_C2, WP_C3, WP_C4};
    float zt0[2 * RAD + 1], zt1[2 * RAD + 1], zx[2 * RAD + 1];
    auto own_plane = [&](int zz, float &v0, float &v1, float &vx) {
        if (!in_grid(G, x, y, zz)) {
            v0 = v1 = vx = 0.f;
            return;
        }
        const long long q = qof(x, y, zz);
        const float azv = T.az[q];
        v0 = azv * t0[q];
        v1 = azv * t1[q];
        vx = x0val(q);
    };
#pragma unroll
    for (int k = 0; k < 2 * RAD; k++) own_plane(z0 - RAD + k, zt0[k], zt1[k], zx[k]);
    float *uo0 = T.u_out + (2 * sh) * T.u_out_ss, *uo1 = T.u_out + (2 * sh + 1) * T.u_out_ss;
    float *do0 = T.d_out + (2 * sh) * T.d_out_ss, *do1 = T.d_out + (2 * sh + 1) * T.d_out_ss;
    const float *di0 = T.d_in + (2 * sh) * T.d_in_ss, *di1 = T.d_in + (2 * sh + 1) * T.d_in_ss;
    for (int z = z0; z < z1; z++) {
        own_plane(z + RAD, zt0[2 * RAD], zt1[2 * RAD], zx[2 * RAD]);
        for (int k = tid; k < TY * WX; k += S::NT) {
            const int ty = k / WX, tx = k - ty * WX;
            const int xx = x0 - RAD + tx, yy = y0 + ty;
            float v0 = 0.f, v1 = 0.f;
            if (in_grid(G, xx, yy, z)) {
                const long long q = qof(xx, yy, z);
                const float axv = T.ax[q];
                v0 = axv * t0[q];
                v1 = axv * t1[q];
            }
            wx0[ty][tx] = v0;
            wx1[ty][tx] = v1;
        }
        if (TY > 1) {
            for (int k = tid; k < WY * TX; k += S::NT) {
                const int ty = k / TX, tx = k - ty * TX;
                const int xx = x0 + tx, yy = y0 - HY + ty;
                float v0 = 0.f, v1 = 0.f;
                if (in_grid(G, xx, yy, z)) {
                    const long long q = qof(xx, yy, z);
                    const float ayv = T.ay[q];
                    v0 = ayv * t0[q];
                    v1 = ayv * t1[q];
                }
                wy0[ty][tx] = v0;
                wy1[ty][tx] = v1;
            }
        }
        for (int k = tid; k < WY * WX; k += S::NT) {
            const int ty = k / WX, tx = k - ty * WX;
            const int xx = x0 - RAD + tx, yy = y0 - HY + ty;
            sx[ty][tx] = in_grid(G, xx, yy, z) ? x0val(qof(xx, yy, z)) : 0.f;
        }
        __syncthreads();
        const long long p = qof(x, y, z);
        if (own) {
            const float c = zx[RAD];
            float hx0 = 0.f, hx1 = 0.f, lx_ = 0.f, hy0 = 0.f, hy1 = 0.f, ly_ = 0.f, hz0 = 0.f, hz1 = 0.f, lz_ = 0.f;
#pragma unroll
            for (int k = 1; k <= RAD; k++) {
                const float cf = cw[k - 1], lf = lw[k - 1];
                hx0 += cf * (wx0[ly][lx + RAD + k] - wx0[ly][lx + RAD - k]);
                hx1 += cf * (wx1[ly][lx + RAD + k] - wx1[ly][lx + RAD - k]);
                lx_ += lf * ((sx[ly + HY][lx + RAD + k] + sx[ly + HY][lx + RAD - k]) - 2.f * c);
                if (TY > 1) {
                    hy0 += cf * (wy0[ly + HY + k][lx] - wy0[ly + HY - k][lx]);
                    hy1 += cf * (wy1[ly + HY + k][lx] - wy1[ly + HY - k][lx]);
                    ly_ += lf * ((sx[ly + HY + k][lx + RAD] + sx[ly + HY - k][lx + RAD]) - 2.f * c);
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
                r0 = T.E[p] * h0p + T.Sd[p] * H1;
                r1 = T.Sd[p] * h0p + H1;
            } else {
                r0 = lap - H0;
                r1 = H1;
            }
            const float bb = T.b[p];
            const float sd = damp_at(G, x, y, z);
            const float cp = 1.f + sd, cm = 1.f - sd;
            const float dn0 = (cm * di0[p] + bb * r0) / cp;
            const float dn1 = (cm * di1[p] + bb * r1) / cp;
            const float un0 = a[p] + dn0, un1 = b[p] + dn1;
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
        } else if (pad && z < G.NZ) {
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
