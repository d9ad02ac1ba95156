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
// Fused into the same launch:
//   - injection of point sources (forward) or of the receiver residual (adjoint): each
//     tile adds its own entries of a CSR table, so no atomics reach global memory;
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

// Increment-form update of one point; returns u^{n+1} and writes the outputs.
template <bool IMG>
__device__ __forceinline__ void update_point(const GridDev &G, const StencilArgs &A, int shot,
                                             long long p, float c, float lap, int x, int y,
                                             int z)
{
    const float a = A.b[p] * lap;
    const float sd = damp_at(G, x, y, z);
    const float din = A.d_in[(long long)shot * A.d_in_ss + p];
    float dn;
    if (sd == 0.f) dn = din + a;
    else dn = ((1.f - sd) * din + a) / (1.f + sd);
    const float un = c + dn;
    A.u_out[(long long)shot * A.u_out_ss + p] = un;
    A.d_out[(long long)shot * A.d_out_ss + p] = dn;
    if (IMG) {
        const long long hp = (long long)shot * A.h_ss + p;
        const float udd = (1.f + sd) * A.h1[hp] - (1.f - sd) * A.h0[hp];
        float *gi = A.img + (long long)shot * A.img_ss + p;
        *gi += A.img_scale * udd * un;
    }
}

// ---------------------------------------------------------------------------------------
// 2-D: 64 x 16 output tile per block, 256 threads, each thread 4 points along z.
// ---------------------------------------------------------------------------------------
template <bool IMG>
__global__ void __launch_bounds__(256) stencil2d_kernel(const GridDev G, const StencilArgs A)
{
    __shared__ float su[T2Z + 2 * RAD][T2X + 2 * RAD];
    __shared__ float sq[T2Z][T2X];
    const int ntx = (G.NX + T2X - 1) / T2X;
    const int ntiles = ntx * ((G.NZ + T2Z - 1) / T2Z);
    if ((int)blockIdx.x >= ntiles) {
        gather_block(A, blockIdx.x - ntiles);
        return;
    }
    const int tile = blockIdx.x, shot = blockIdx.y, tid = threadIdx.x;
    const int x0 = (tile % ntx) * T2X, z0 = (tile / ntx) * T2Z;
    const float *__restrict__ u = A.u_in + (long long)shot * A.u_in_ss;
    const int lx = tid & 63;

    for (int row = tid >> 6; row < T2Z + 2 * RAD; row += 4) {
        const int gz = z0 + row - RAD;
        const bool zin = gz >= 0 && gz < G.NZ;
        const long long rowp = (long long)gz * G.NX;
        const int gx = x0 + lx;
        su[row][lx + RAD] = (zin && gx < G.NX) ? u[rowp + gx] : 0.f;
        if (lx < 2 * RAD) {
            const int hc = lx < RAD ? lx : T2X + lx;
            const int hgx = x0 + hc - RAD;
            su[row][hc] = (zin && hgx >= 0 && hgx < G.NX) ? u[rowp + hgx] : 0.f;
        }
    }
    int e0 = 0, e1 = 0;
    if (A.inj) {
        const int *off = A.inj_off + (long long)shot * (ntiles + 1);
        e0 = off[tile];
        e1 = off[tile + 1];
    }
    if (e1 > e0) {
        for (int i = tid; i < T2Z * T2X; i += 256) (&sq[0][0])[i] = 0.f;
        __syncthreads();
        const float *tr = A.traces + (long long)shot * A.tr_ss + (long long)A.step * A.tr_ts;
        for (int e = e0 + tid; e < e1; e += 256) {
            const InjEntry E = A.inj[e];
            atomicAdd(&(&sq[0][0])[E.a], E.w * A.tr_sign * tr[(long long)E.trace * A.tr_rs]);
        }
    }
    __syncthreads();

    const int gx = x0 + lx;
    if (gx >= G.NX) return;
#pragma unroll
    for (int k = 0; k < T2Z / 4; k++) {
        const int lz = (tid >> 6) + 4 * k;
        const int gz = z0 + lz;
        if (gz >= G.NZ) break;
        const int sr = lz + RAD, sc = lx + RAD;
        const float c = su[sr][sc];
        const float lxx = WP_C1 * ((su[sr][sc + 1] - c) + (su[sr][sc - 1] - c)) +
                          WP_C2 * ((su[sr][sc + 2] - c) + (su[sr][sc - 2] - c)) +
                          WP_C3 * ((su[sr][sc + 3] - c) + (su[sr][sc - 3] - c)) +
                          WP_C4 * ((su[sr][sc + 4] - c) + (su[sr][sc - 4] - c));
        const float lzz = WP_C1 * ((su[sr + 1][sc] - c) + (su[sr - 1][sc] - c)) +
                          WP_C2 * ((su[sr + 2][sc] - c) + (su[sr - 2][sc] - c)) +
                          WP_C3 * ((su[sr + 3][sc] - c) + (su[sr - 3][sc] - c)) +
                          WP_C4 * ((su[sr + 4][sc] - c) + (su[sr - 4][sc] - c));
        float lap = G.ihx2 * lxx + G.ihz2 * lzz;
        if (e1 > e0) lap += sq[lz][lx];
        update_point<IMG>(G, A, shot, (long long)gz * G.NX + gx, c, lap, gx, 0, gz);
    }
}

// ---------------------------------------------------------------------------------------
// 3-D: a 32 x 16 (x, y) block of columns marches T3Z planes along z.  Each thread keeps
// the 9 z-neighbours of its column in registers; the current plane (with x/y halos) sits
// in shared memory.
// ---------------------------------------------------------------------------------------
template <bool IMG>
__global__ void __launch_bounds__(512) stencil3d_kernel(const GridDev G, const StencilArgs A)
{
    __shared__ float sp[T3Y + 2 * RAD][T3X + 2 * RAD];
    __shared__ float sq[T3Y][T3X];
    const int ntx = (G.NX + T3X - 1) / T3X, nty = (G.NY + T3Y - 1) / T3Y;
    const int ntiles = ntx * nty * ((G.NZ + T3Z - 1) / T3Z);
    if ((int)blockIdx.x >= ntiles) {
        gather_block(A, blockIdx.x - ntiles);
        return;
    }
    const int tile = blockIdx.x, shot = blockIdx.y, tid = threadIdx.x;
    const int x0 = (tile % ntx) * T3X, y0 = ((tile / ntx) % nty) * T3Y;
    const int z0 = (tile / (ntx * nty)) * T3Z;
    const int z1 = min(z0 + T3Z, G.NZ);
    const int lx = tid & (T3X - 1), ly = tid / T3X;
    const int gx = x0 + lx, gy = y0 + ly;
    const bool inside = gx < G.NX && gy < G.NY;
    const long long PS = (long long)G.NX * G.NY;
    const float *__restrict__ u = A.u_in + (long long)shot * A.u_in_ss;
    const long long col = (long long)gy * G.NX + gx;

    auto ld = [&](int x, int y, int z) -> float {
        return (x >= 0 && x < G.NX && y >= 0 && y < G.NY && z >= 0 && z < G.NZ)
                   ? u[(long long)z * PS + (long long)y * G.NX + x]
                   : 0.f;
    };
    float q[2 * RAD + 1];
#pragma unroll
    for (int k = 0; k < 2 * RAD; k++) {
        const int z = z0 - RAD + k;
        q[k] = (inside && z >= 0 && z < G.NZ) ? u[(long long)z * PS + col] : 0.f;
    }
    const int *off = A.inj ? A.inj_off + (long long)shot * ((long long)ntiles * T3Z + 1) : nullptr;
    const float *tr = A.inj ? A.traces + (long long)shot * A.tr_ss + (long long)A.step * A.tr_ts
                            : nullptr;

    for (int z = z0; z < z1; z++) {
        q[2 * RAD] = (inside && z + RAD < G.NZ) ? u[(long long)(z + RAD) * PS + col] : 0.f;
        __syncthreads();
        sp[ly + RAD][lx + RAD] = q[RAD];
        if (lx < RAD) sp[ly + RAD][lx] = ld(gx - RAD, gy, z);
        if (lx >= T3X - RAD) sp[ly + RAD][lx + 2 * RAD] = ld(gx + RAD, gy, z);
        if (ly < RAD) sp[ly][lx + RAD] = ld(gx, gy - RAD, z);
        if (ly >= T3Y - RAD) sp[ly + 2 * RAD][lx + RAD] = ld(gx, gy + RAD, z);
        int e0 = 0, e1 = 0;
        if (off) {
            const long long key = (long long)tile * T3Z + (z - z0);
            e0 = off[key];
            e1 = off[key + 1];
        }
        if (e1 > e0) {
            sq[ly][lx] = 0.f;
            __syncthreads();
            for (int e = e0 + tid; e < e1; e += T3X * T3Y) {
                const InjEntry E = A.inj[e];
                atomicAdd(&(&sq[0][0])[E.a], E.w * A.tr_sign * tr[(long long)E.trace * A.tr_rs]);
            }
        }
        __syncthreads();
        if (inside) {
            const int sr = ly + RAD, sc = lx + RAD;
            const float c = q[RAD];
            const float lxx = WP_C1 * ((sp[sr][sc + 1] - c) + (sp[sr][sc - 1] - c)) +
                              WP_C2 * ((sp[sr][sc + 2] - c) + (sp[sr][sc - 2] - c)) +
                              WP_C3 * ((sp[sr][sc + 3] - c) + (sp[sr][sc - 3] - c)) +
                              WP_C4 * ((sp[sr][sc + 4] - c) + (sp[sr][sc - 4] - c));
            const float lyy = WP_C1 * ((sp[sr + 1][sc] - c) + (sp[sr - 1][sc] - c)) +
                              WP_C2 * ((sp[sr + 2][sc] - c) + (sp[sr - 2][sc] - c)) +
                              WP_C3 * ((sp[sr + 3][sc] - c) + (sp[sr - 3][sc] - c)) +
                              WP_C4 * ((sp[sr + 4][sc] - c) + (sp[sr - 4][sc] - c));
            const float lzz = WP_C1 * ((q[RAD + 1] - c) + (q[RAD - 1] - c)) +
                              WP_C2 * ((q[RAD + 2] - c) + (q[RAD - 2] - c)) +
                              WP_C3 * ((q[RAD + 3] - c) + (q[RAD - 3] - c)) +
                              WP_C4 * ((q[RAD + 4] - c) + (q[RAD - 4] - c));
            float lap = G.ihx2 * lxx + G.ihy2 * lyy + G.ihz2 * lzz;
            if (e1 > e0) lap += sq[ly][lx];
            update_point<IMG>(G, A, shot, (long long)z * PS + col, c, lap, gx, gy, z);
        }
#pragma unroll
        for (int k = 0; k < 2 * RAD; k++) q[k] = q[k + 1];
    }
}

__global__ void gather_kernel(const StencilArgs A) { gather_block(A, blockIdx.x); }

cudaError_t launch_stencil(const GridDev &G, const StencilArgs &A, bool imaging, cudaStream_t s)
{
    const int ng = A.do_gather ? (A.nrec + 255) / 256 : 0;
    cudaEvent_t ev = prof_begin(PROF_STENCIL, s);
    if (G.ndim == 2) {
        dim3 grid(tiles2d(G) + ng, A.nshots);
        if (imaging) stencil2d_kernel<true><<<grid, 256, 0, s>>>(G, A);
        else stencil2d_kernel<false><<<grid, 256, 0, s>>>(G, A);
    } else {
        StencilArgs B = A;
        const int ng3 = A.do_gather ? (A.nrec + 511) / 512 : 0;
        dim3 grid(tiles3d(G) + ng3, A.nshots);
        if (imaging) stencil3d_kernel<true><<<grid, 512, 0, s>>>(G, B);
        else stencil3d_kernel<false><<<grid, 512, 0, s>>>(G, B);
    }
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
