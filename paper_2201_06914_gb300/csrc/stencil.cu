// Acoustic time-step kernels (forward and adjoint use the same kernel, Sec. 2.2).
//
// One launch advances every shot of a batch by one leapfrog step of
//   m (u_tt + sigma u_t) - Laplacian(u) = q
// written in increment form to limit FP32 rounding growth: with d^n = u^n - u^{n-1},
//   a^n     = (dt^2/m) (L u^n + q^n)                  (= dt^2 * u_tt^n)
//   d^{n+1} = ((1 - sigma dt/2) d^n + a^n) / (1 + sigma dt/2)
//   u^{n+1} = u^n + d^{n+1}
// which is algebraically the centred scheme (1+sigma dt/2)u^{n+1} - 2u^n +
// (1-sigma dt/2)u^{n-1} = a^n.  L is the 8th-order Laplacian evaluated in difference
// form, sum_k c_k ((u[+k] - u[0]) + (u[-k] - u[0])), with zero values beyond the grid.
//
// Data movement: a block owns a TX x TY patch of (x, y) columns and marches `tz` planes
// along z.  Each thread keeps the 9 z-neighbours of its column in registers (every u value
// is read from memory once per block, plus an 8-plane z-halo per march); the current plane
// with its x/y halos sits in a double-buffered shared-memory plane, so one barrier per
// plane suffices.  The increment and dt^2/m of a point are loaded before the barrier.
//
// Fused into the same launch:
//   - injection of point sources (forward) or of the receiver residual (adjoint): each
//     block adds the entries of its (tile, plane) keys from a CSR table in shared memory,
//     so no atomics reach global memory;
//   - recording d = R u^n of the input wavefield (extra blocks after the stencil tiles);
//   - the exact imaging condition of Eq. 2 (template flag IMG): g += u_tt^j * v^j with
//     u_tt^j rebuilt from two stored forward increments.
#include "wp_internal.cuh"

namespace wp {

__device__ __forceinline__ void gather_block(const StencilArgs &A, int gblock)
{
    const int shot = blockIdx.y;
    const int rec = gblock * blockDim.x + threadIdx.x;
    if (rec >= A.nrec) return;
    const float *u = A.u_in + (long long)shot * A.u_in_ss;
    const long long base = ((long long)shot * A.nrec + rec) * A.ncorner;
    float acc = 0.f;
    for (int c = 0; c < A.ncorner; c++) acc += A.g_w[base + c] * u[A.g_idx[base + c]];
    A.g_out[(long long)shot * A.g_ss + (long long)A.g_row * A.nrec + rec] = acc;
}

__device__ __forceinline__ float d2(float c, float p1, float m1, float p2, float m2, float p3,
                                    float m3, float p4, float m4)
{
    return WP_C1 * ((p1 - c) + (m1 - c)) + WP_C2 * ((p2 - c) + (m2 - c)) +
           WP_C3 * ((p3 - c) + (m3 - c)) + WP_C4 * ((p4 - c) + (m4 - c));
}

// One block: TXT x TY threads, each owning VX columns (x = x0 + lx + v*TXT); the tile is
// TX = TXT*VX columns wide.  The z-march is unrolled nine times so that the 9-deep
// register queue rotates by renaming instead of moving values.
template <int TXT, int TY, bool IMG>
struct March {
    static constexpr int TX = TXT * VX;
    static constexpr int HY = TY > 1 ? RAD : 0;
    static constexpr int NT = TXT * TY;
    static constexpr int W = TX + 2 * RAD;   // shared plane row length

    const GridDev &G;
    const StencilArgs &A;
    float (*sp)[TY + 2 * HY][W];
    float (*sq)[TY][TX];
    int tid, lx, ly, gy, x0, z0, z1, tile, shot, PS, col0;
    bool in_y;
    bool in_x[VX];
    const float *u, *dinp, *bp;
    float *uo, *dout;
    float *imgp;
    const float *h1p, *h0p;
    const int *off;
    const float *tr;
    bool tile_inj, interior_xy;
    float sdxy[VX];
    // x/y halo role of this thread
    bool hxl, hxr, hyl, hyr;
    int hxx, hyy;
    // values of the next plane fetched one plane ahead
    float nhx, nhy[VX], ndin[VX], nbb[VX];
    float q[VX][9];

    __device__ __forceinline__ float ld(int x, int y, int z) const
    {
        return (x >= 0 && x < G.NX && y >= 0 && y < G.NY) ? u[z * PS + y * G.NX + x] : 0.f;
    }

    __device__ __forceinline__ void fetch(int z)
    {
        nhx = (hxl || hxr) ? ld(hxx, gy, z) : 0.f;
#pragma unroll
        for (int v = 0; v < VX; v++) {
            const int x = x0 + lx + v * TXT;
            nhy[v] = (hyl || hyr) ? ld(x, hyy, z) : 0.f;
            const int p = z * PS + col0 + v * TXT;
            ndin[v] = (in_y && in_x[v]) ? dinp[p] : 0.f;
            nbb[v] = (in_y && in_x[v]) ? bp[p] : 0.f;
        }
    }

    template <int R>
    __device__ __forceinline__ void step(int z)
    {
        const int buf = (z - z0) & 1;
        float(*P)[W] = sp[buf];
#pragma unroll
        for (int v = 0; v < VX; v++)
            q[v][(8 + R) % 9] = (in_y && in_x[v] && z + RAD < G.NZ) ? u[(z + RAD) * PS + col0 + v * TXT] : 0.f;
        const float hx = nhx;
        float hy[VX], din[VX], bb[VX];
#pragma unroll
        for (int v = 0; v < VX; v++) {
            hy[v] = nhy[v];
            din[v] = ndin[v];
            bb[v] = nbb[v];
        }
        if (z + 1 < z1) fetch(z + 1);
#pragma unroll
        for (int v = 0; v < VX; v++) P[ly + HY][lx + v * TXT + RAD] = q[v][(4 + R) % 9];
        if (hxl) P[ly + HY][lx] = hx;
        if (hxr) P[ly + HY][lx + TX - TXT + 2 * RAD] = hx;
        if (TY > 1) {
#pragma unroll
            for (int v = 0; v < VX; v++) {
                if (hyl) P[ly][lx + v * TXT + RAD] = hy[v];
                if (hyr) P[ly + 2 * HY][lx + v * TXT + RAD] = hy[v];
            }
        }
        int e0 = 0, e1 = 0;
        if (tile_inj) {
            const long long key = (long long)tile * G.tz + (z - z0);
            e0 = off[key];
            e1 = off[key + 1];
        }
        if (e1 > e0) {
#pragma unroll
            for (int v = 0; v < VX; v++) sq[buf][ly][lx + v * TXT] = 0.f;
            __syncthreads();
            for (int e = e0 + tid; e < e1; e += NT) {
                const InjEntry E = A.inj[e];
                atomicAdd(&(&sq[buf][0][0])[E.a], E.w * A.tr_sign * tr[(long long)E.trace * A.tr_rs]);
            }
        }
        __syncthreads();
        const float sdz = damp_term(z, G.nz, G.nbl, G.hs0z, G.inv_nbl);
        const bool fast = interior_xy && sdz == 0.f;
#pragma unroll
        for (int v = 0; v < VX; v++) {
            if (!(in_y && in_x[v])) continue;
            const int sr = ly + HY, sc = lx + v * TXT + RAD;
            const float c = q[v][(4 + R) % 9];
            float lap = G.ihx2 * (WP_C1 * ((P[sr][sc + 1] - c) + (P[sr][sc - 1] - c)) +
                                  WP_C2 * ((P[sr][sc + 2] - c) + (P[sr][sc - 2] - c)) +
                                  WP_C3 * ((P[sr][sc + 3] - c) + (P[sr][sc - 3] - c)) +
                                  WP_C4 * ((P[sr][sc + 4] - c) + (P[sr][sc - 4] - c)));
            if (TY > 1)
                lap += G.ihy2 * (WP_C1 * ((P[sr + 1][sc] - c) + (P[sr - 1][sc] - c)) +
                                 WP_C2 * ((P[sr + 2][sc] - c) + (P[sr - 2][sc] - c)) +
                                 WP_C3 * ((P[sr + 3][sc] - c) + (P[sr - 3][sc] - c)) +
                                 WP_C4 * ((P[sr + 4][sc] - c) + (P[sr - 4][sc] - c)));
            lap += G.ihz2 * (WP_C1 * ((q[v][(5 + R) % 9] - c) + (q[v][(3 + R) % 9] - c)) +
                             WP_C2 * ((q[v][(6 + R) % 9] - c) + (q[v][(2 + R) % 9] - c)) +
                             WP_C3 * ((q[v][(7 + R) % 9] - c) + (q[v][(1 + R) % 9] - c)) +
                             WP_C4 * ((q[v][(8 + R) % 9] - c) + (q[v][(0 + R) % 9] - c)));
            if (e1 > e0) lap += sq[buf][ly][lx + v * TXT];
            const float a = bb[v] * lap;
            float dn, sd = 0.f;
            if (fast) {
                dn = din[v] + a;
            } else {
                sd = sdxy[v] + sdz;
                dn = (sd == 0.f) ? din[v] + a : ((1.f - sd) * din[v] + a) * __frcp_rn(1.f + sd);
            }
            const float un = c + dn;
            const int p = z * PS + col0 + v * TXT;
            uo[p] = un;
            dout[p] = dn;
            if (IMG) {
                const float udd = (1.f + sd) * h1p[p] - (1.f - sd) * h0p[p];
                imgp[p] += A.img_scale * udd * un;
            }
        }
    }
};

template <int TXT, int TY, bool IMG>
__global__ void __launch_bounds__(TXT *TY, (TY > 1 ? 1 : 6)) march_kernel(const GridDev G, const StencilArgs A)
{
    using M = March<TXT, TY, IMG>;
    __shared__ float sp[2][TY + 2 * M::HY][M::W];
    __shared__ float sq[2][TY][M::TX];
    const int ntx = (G.NX + M::TX - 1) / M::TX, nty = (G.NY + TY - 1) / TY;
    const int ntiles = ntx * nty * ((G.NZ + G.tz - 1) / G.tz);
    if ((int)blockIdx.x >= ntiles) {
        gather_block(A, blockIdx.x - ntiles);
        return;
    }
    M m{G, A};
    m.sp = sp;
    m.sq = sq;
    m.tid = threadIdx.x;
    m.tile = blockIdx.x;
    m.shot = blockIdx.y;
    m.lx = m.tid % TXT;
    m.ly = m.tid / TXT;
    m.x0 = (m.tile % ntx) * M::TX;
    const int y0 = ((m.tile / ntx) % nty) * TY;
    m.z0 = (m.tile / (ntx * nty)) * G.tz;
    m.z1 = min(m.z0 + G.tz, G.NZ);
    m.gy = y0 + m.ly;
    m.in_y = m.gy < G.NY;
    m.PS = G.NX * G.NY;
    m.col0 = m.gy * G.NX + m.x0 + m.lx;
    const long long sh = m.shot;
    m.u = A.u_in + sh * A.u_in_ss;
    m.dinp = A.d_in + sh * A.d_in_ss;
    m.bp = A.b;
    m.uo = A.u_out + sh * A.u_out_ss;
    m.dout = A.d_out + sh * A.d_out_ss;
    if (IMG) {
        m.imgp = A.img + sh * A.img_ss;
        m.h1p = A.h1 + sh * A.h_ss;
        m.h0p = A.h0 + sh * A.h_ss;
    }
    m.off = A.inj ? A.inj_off + sh * ((long long)ntiles * G.tz + 1) : nullptr;
    m.tile_inj = m.off && m.off[(long long)m.tile * G.tz] < m.off[(long long)m.tile * G.tz + (m.z1 - m.z0)];
    m.tr = m.tile_inj ? A.traces + sh * A.tr_ss + (long long)A.step * A.tr_ts : nullptr;
    m.interior_xy = m.x0 >= G.nbl && m.x0 + M::TX <= G.nbl + G.nx &&
                    (TY == 1 || (y0 >= G.nbl && y0 + TY <= G.nbl + G.ny));
#pragma unroll
    for (int v = 0; v < VX; v++) {
        const int x = m.x0 + m.lx + v * TXT;
        m.in_x[v] = x < G.NX;
        m.sdxy[v] = damp_term(x, G.nx, G.nbl, G.hs0x, G.inv_nbl) +
                    (TY > 1 ? damp_term(m.gy, G.ny, G.nbl, G.hs0y, G.inv_nbl) : 0.f);
    }
    m.hxl = m.lx < RAD;
    m.hxr = m.lx >= TXT - RAD;
    m.hxx = m.hxl ? m.x0 - RAD + m.lx : m.x0 + M::TX + (m.lx - (TXT - RAD));
    m.hyl = TY > 1 && m.ly < M::HY;
    m.hyr = TY > 1 && m.ly >= TY - M::HY;
    m.hyy = m.hyl ? m.gy - M::HY : m.gy + M::HY;
#pragma unroll
    for (int v = 0; v < VX; v++) {
#pragma unroll
        for (int k = 0; k < 2 * RAD; k++) {
            const int z = m.z0 - RAD + k;
            m.q[v][k] = (m.in_y && m.in_x[v] && z >= 0 && z < G.NZ) ? m.u[z * m.PS + m.col0 + v * TXT] : 0.f;
        }
    }
    m.fetch(m.z0);
    for (int z = m.z0; z < m.z1; z += 9) {
        m.template step<0>(z);
        if (z + 1 < m.z1) m.template step<1>(z + 1); else break;
        if (z + 2 < m.z1) m.template step<2>(z + 2); else break;
        if (z + 3 < m.z1) m.template step<3>(z + 3); else break;
        if (z + 4 < m.z1) m.template step<4>(z + 4); else break;
        if (z + 5 < m.z1) m.template step<5>(z + 5); else break;
        if (z + 6 < m.z1) m.template step<6>(z + 6); else break;
        if (z + 7 < m.z1) m.template step<7>(z + 7); else break;
        if (z + 8 < m.z1) m.template step<8>(z + 8); else break;
    }
}

__global__ void gather_kernel(const StencilArgs A) { gather_block(A, blockIdx.x); }

template <int TXT, int TY>
static void launch_march(const GridDev &G, const StencilArgs &A, bool imaging, cudaStream_t s)
{
    constexpr int NT = TXT * TY;
    const int ng = A.do_gather ? (A.nrec + NT - 1) / NT : 0;
    dim3 grid(stencil_tiles(G) + ng, A.nshots);
    if (imaging) march_kernel<TXT, TY, true><<<grid, NT, 0, s>>>(G, A);
    else march_kernel<TXT, TY, false><<<grid, NT, 0, s>>>(G, A);
}

cudaError_t launch_stencil(const GridDev &G, const StencilArgs &A, bool imaging, cudaStream_t s)
{
    cudaEvent_t ev = prof_begin(PROF_STENCIL, s);
    if (G.ndim == 2) launch_march<T2TX, T2Y>(G, A, imaging, s);
    else launch_march<T3TX, T3Y>(G, A, imaging, s);
    prof_end(PROF_STENCIL, ev, s);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_gather(const GridDev &G, const StencilArgs &A, cudaStream_t s)
{
    (void)G;
    dim3 grid((A.nrec + 255) / 256, A.nshots);
    gather_kernel<<<grid, 256, 0, s>>>(A);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
