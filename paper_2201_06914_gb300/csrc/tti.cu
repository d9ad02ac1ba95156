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
// to the updated increments and fields.
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

__device__ __forceinline__ bool inside(const GridDev &G, int x, int y, int z)
{
    return x >= 0 && x < G.NX && y >= 0 && y < G.NY && z >= 0 && z < G.NZ;
}

// Input field j (0, 1) of the step at padded point q: forward the fields themselves,
// adjoint the combinations e = E a + S b, f = S a + b.
__device__ __forceinline__ float xin(const TtiArgs &T, const float *a, const float *b, int j,
                                     long long q)
{
    if (!T.adjoint) return j == 0 ? a[q] : b[q];
    const float av = a[q], bv = b[q];
    return j == 0 ? T.E[q] * av + T.Sd[q] * bv : T.Sd[q] * av + bv;
}

}  // namespace

// Pass 1: t_j = Dr x_j = sum_i a_i D_i x_j for both fields of every shot.
__global__ void tti_pass1_kernel(const GridDev G, const TtiArgs T)
{
    const long long sh = blockIdx.y;
    const float *a = T.u_in + (2 * sh) * T.u_in_ss;
    const float *b = T.u_in + (2 * sh + 1) * T.u_in_ss;
    float *t0 = T.t + (2 * sh) * T.t_ss, *t1 = T.t + (2 * sh + 1) * T.t_ss;
    const float ih[3] = {1.f / G.hx, 1.f / G.hy, 1.f / G.hz};
    const long long st[3] = {1, G.NXp, (long long)G.NXp * G.NY};
    const float cw[4] = {D1C1, D1C2, D1C3, D1C4};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < G.Np;
         p += (long long)gridDim.x * blockDim.x) {
        const Pt c = coords(G, p);
        if (c.x >= G.NX) {
            t0[p] = 0.f;
            t1[p] = 0.f;
            continue;
        }
        float acc0 = 0.f, acc1 = 0.f;
        const float ai[3] = {T.ax[p], G.ndim == 3 ? T.ay[p] : 0.f, T.az[p]};
        for (int i = 0; i < 3; i++) {
            if (i == 1 && G.ndim == 2) continue;
            float d0 = 0.f, d1 = 0.f;
            for (int k = 1; k <= RAD; k++) {
                const int xp = c.x + (i == 0 ? k : 0), yp = c.y + (i == 1 ? k : 0), zp = c.z + (i == 2 ? k : 0);
                const int xm = c.x - (i == 0 ? k : 0), ym = c.y - (i == 1 ? k : 0), zm = c.z - (i == 2 ? k : 0);
                const bool ip = inside(G, xp, yp, zp), im = inside(G, xm, ym, zm);
                const long long qp = p + k * st[i], qm = p - k * st[i];
                const float p0 = ip ? xin(T, a, b, 0, qp) : 0.f, m0 = im ? xin(T, a, b, 0, qm) : 0.f;
                const float p1 = ip ? xin(T, a, b, 1, qp) : 0.f, m1 = im ? xin(T, a, b, 1, qm) : 0.f;
                d0 += cw[k - 1] * (p0 - m0);
                d1 += cw[k - 1] * (p1 - m1);
            }
            acc0 += ai[i] * d0 * ih[i];
            acc1 += ai[i] * d1 * ih[i];
        }
        t0[p] = acc0;
        t1[p] = acc1;
    }
}

// Pass 2: Hz_j = sum_i D_i (a_i t_j), L x_0, combination, leapfrog update of both fields.
template <bool IMG>
__global__ void tti_pass2_kernel(const GridDev G, const TtiArgs T)
{
    const long long sh = blockIdx.y;
    const float *a = T.u_in + (2 * sh) * T.u_in_ss;
    const float *b = T.u_in + (2 * sh + 1) * T.u_in_ss;
    const float *t0 = T.t + (2 * sh) * T.t_ss, *t1 = T.t + (2 * sh + 1) * T.t_ss;
    const float ih[3] = {1.f / G.hx, 1.f / G.hy, 1.f / G.hz};
    const float ih2[3] = {G.ihx2, G.ihy2, G.ihz2};
    const long long st[3] = {1, G.NXp, (long long)G.NXp * G.NY};
    const float cw[4] = {D1C1, D1C2, D1C3, D1C4};
    const float lw[4] = {WP_C1, WP_C2, WP_C3, WP_C4};
    const float *aw[3] = {T.ax, T.ay, T.az};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < G.Np;
         p += (long long)gridDim.x * blockDim.x) {
        const Pt c = coords(G, p);
        float *uo0 = T.u_out + (2 * sh) * T.u_out_ss, *uo1 = T.u_out + (2 * sh + 1) * T.u_out_ss;
        float *do0 = T.d_out + (2 * sh) * T.d_out_ss, *do1 = T.d_out + (2 * sh + 1) * T.d_out_ss;
        if (c.x >= G.NX) {
            uo0[p] = 0.f;
            uo1[p] = 0.f;
            do0[p] = 0.f;
            do1[p] = 0.f;
            continue;
        }
        const float x0c = xin(T, a, b, 0, p);
        float hz0 = 0.f, hz1 = 0.f, lap = 0.f;
        for (int i = 0; i < 3; i++) {
            if (i == 1 && G.ndim == 2) continue;
            float h0 = 0.f, h1 = 0.f, l = 0.f;
            for (int k = 1; k <= RAD; k++) {
                const int xp = c.x + (i == 0 ? k : 0), yp = c.y + (i == 1 ? k : 0), zp = c.z + (i == 2 ? k : 0);
                const int xm = c.x - (i == 0 ? k : 0), ym = c.y - (i == 1 ? k : 0), zm = c.z - (i == 2 ? k : 0);
                const bool ip = inside(G, xp, yp, zp), im = inside(G, xm, ym, zm);
                const long long qp = p + k * st[i], qm = p - k * st[i];
                const float ap = ip ? aw[i][qp] : 0.f, am = im ? aw[i][qm] : 0.f;
                h0 += cw[k - 1] * ((ip ? ap * t0[qp] : 0.f) - (im ? am * t0[qm] : 0.f));
                h1 += cw[k - 1] * ((ip ? ap * t1[qp] : 0.f) - (im ? am * t1[qm] : 0.f));
                const float xp0 = ip ? xin(T, a, b, 0, qp) : 0.f, xm0 = im ? xin(T, a, b, 0, qm) : 0.f;
                l += lw[k - 1] * ((xp0 + xm0) - 2.f * x0c);
            }
            hz0 += h0 * ih[i];
            hz1 += h1 * ih[i];
            lap += l * ih2[i];
        }
        float r0, r1;
        if (!T.adjoint) {
            const float h0p = lap - hz0;
            r0 = T.E[p] * h0p + T.Sd[p] * hz1;
            r1 = T.Sd[p] * h0p + hz1;
        } else {
            r0 = lap - hz0;
            r1 = hz1;
        }
        const float bb = T.b[p];
        const float sd = damp_at(G, c.x, c.y, c.z);
        const float cp = 1.f + sd, cm = 1.f - sd;
        const float *di0 = T.d_in + (2 * sh) * T.d_in_ss, *di1 = T.d_in + (2 * sh + 1) * T.d_in_ss;
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

cudaError_t launch_tti_step(const GridDev &G, const TtiArgs &T, const TtiInject &J, cudaStream_t s)
{
    dim3 grid(blocks_for(G.Np), T.nshots);
    cudaEvent_t ev = prof_begin(PROF_STENCIL, s);
    tti_pass1_kernel<<<grid, 256, 0, s>>>(G, T);
    if (T.img) tti_pass2_kernel<true><<<grid, 256, 0, s>>>(G, T);
    else tti_pass2_kernel<false><<<grid, 256, 0, s>>>(G, T);
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
