// One time step of the isotropic scheme at four adjacent columns, shared by the
// single-step (stencil.cu) and two-step (stencil2.cu) kernels so that both perform the
// same operations in the same order and give the same bits.
//
// The arithmetic runs on pairs of columns with the packed FP32 instructions of sm_100+
// (add/sub/mul/fma .rn.f32x2: each lane is the IEEE single-precision operation with
// round-to-nearest), which halves the instruction count of the Laplacian.
//
// Laplacian in pairwise form with the axes merged (Sec. 2.1, space order 8):
//   L u = (1/hx^2) sum_k c_k ( (u[x+k] + u[x-k]) + rz (u[z+k] + u[z-k]) + ry (u[y+k] + u[y-k])
//                              - 2 (1 + rz + ry) u )
// with rz = hx^2/hz^2, ry = hx^2/hy^2.  Neighbour pairs are summed first and the centre is
// removed per offset, which keeps the FP32 rounding of L u at the level of the fully
// differenced form (the plain sum c_0 u + sum c_k (u[+k] + u[-k]) loses about a digit on
// smooth fields).  Then, with s = sigma dt / 2 and b = dt^2 / m, the (u, d) form (adjoint)
//   d^{n+1} = d^n + b (L u + q)                               (s = 0)
//   d^{n+1} = ((1 - s) d^n + b (L u + q)) * rcp(1 + s)        (absorbing layer)
//   u^{n+1} = u^n + d^{n+1}
// or the (w, d) form (forward), whose state is w^{n-1} = L u^{n-1} and d^n = u^n - u^{n-1}
// and which never forms u:
//   w^n     = w^{n-1} + L d^n
//   d^{n+1} = d^n + b (w^n + q)                               (s = 0)
//   d^{n+1} = ((1 - s) d^n + b (w^n + q)) * rcp(1 + s)        (absorbing layer)
// Both are the same recurrence in exact arithmetic (L is linear).  In FP32 the (w, d) form
// never rounds u itself: the (u, d) form adds d to a much larger u every step, and L
// amplifies that rounding noise (white in space) far more than it amplifies the wave, so
// u_tt = b (w + q) / dt^2, which the forward's probe projections are built from, is
// several times more accurate in the (w, d) form (2.9e-6 instead of 1.5e-5 relative L2
// for P_u after 1000 steps of the two-layer 201 x 201 workload, FP32 emulation on the
// CPU).  The adjoint keeps the (u, d) form: its projections use v itself, not a second
// derivative.
//
// In both forms the field that the stencil reads with halos ("X": u, or d) and the field
// read only at the own point ("Y": d, or w) enter and leave through the same arguments:
// cc/wz = X^n, din = Y^n, un = X^{n+1}, dn = Y^{n+1}.
#pragma once

#include "wp_internal.cuh"

namespace wp {
namespace step {

typedef unsigned long long f2;   // two floats in one 64-bit register (low word first)

struct __align__(16) P4 {        // four adjacent columns as two pairs
    f2 a, b;                     // columns (0, 1) and (2, 3)
};

__device__ __forceinline__ f2 pk(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2 dup(float v) { return pk(v, v); }

__device__ __forceinline__ P4 lds(uint32_t addr)
{
    P4 v;
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(v.a), "=l"(v.b) : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts(uint32_t addr, const P4 &v)
{
    asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(addr), "l"(v.a), "l"(v.b) : "memory");
}
__device__ __forceinline__ P4 zero() { return P4{0ull, 0ull}; }

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ const f2 &half(const P4 &v, int p) { return p == 0 ? v.a : v.b; }

// Columns i and i+1 of the 12 x-neighbour values wl | centre | wr (i in 0..10).
__device__ __forceinline__ f2 xpair(const P4 &wl, const P4 &cc, const P4 &wr, int i)
{
    const P4 &q = i < 4 ? wl : i < 8 ? cc : wr;
    if ((i & 1) == 0) return half(q, (i & 3) >> 1);
    float w[12];
    upk(wl.a, w[0], w[1]);
    upk(wl.b, w[2], w[3]);
    upk(cc.a, w[4], w[5]);
    upk(cc.b, w[6], w[7]);
    upk(wr.a, w[8], w[9]);
    upk(wr.b, w[10], w[11]);
    return pk(w[i], w[i + 1]);
}

// One step at the four columns of the thread.  wz: own column z window with the centre at
// wz[RAD]; wy_p / wy_m: y neighbours +k / -k (3-D only, Y = true); wl / wr: x neighbours
// (columns -4..-1 and +4..+7); sqv: injected terms of the four columns (read if inj);
// sdx: absorbing-layer term of the columns along x (and y); z: plane index.  Returns the
// new increment and field; sdv receives the absorbing term of each column (0 inside).
template <bool Y, bool WD = false>
__device__ __forceinline__ void step4(const P4 *wz, const P4 *wy_p, const P4 *wy_m, const P4 &wl,
                                      const P4 &wr, const P4 &din, const P4 &bb, const float *sqv,
                                      bool inj, bool interior, const float sdx[4], int z,
                                      const GridDev &G, P4 &dn, P4 &un, float sdv[4])
{
    const P4 &cc = wz[RAD];
    const f2 rz = dup(G.lrz), ry = dup(G.lry), nkc0 = dup(-G.lapK), ihx2 = dup(G.ihx2);
    f2 lap[2], wn[2];
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const int j = 2 * p;
        const f2 c = half(cc, p);
        f2 acc = 0ull;
#pragma unroll
        for (int k = 1; k <= RAD; k++) {
            f2 sp = add2(xpair(wl, cc, wr, 4 + j + k), xpair(wl, cc, wr, 4 + j - k));
            sp = fma2(rz, add2(half(wz[RAD + k], p), half(wz[RAD - k], p)), sp);
            if (Y) sp = fma2(ry, add2(half(wy_p[k - 1], p), half(wy_m[k - 1], p)), sp);
            const f2 ck = dup(k == 1 ? WP_C1 : k == 2 ? WP_C2 : k == 3 ? WP_C3 : WP_C4);
            // centre removed with one rounding: sp - 2 (1 + rz + ry) u (the neighbour sum and
            // the centre term nearly cancel on smooth fields)
            const f2 t = fma2(nkc0, c, sp);
            acc = k == 1 ? mul2(ck, t) : fma2(ck, t, acc);
        }
        lap[p] = mul2(ihx2, acc);
        if (WD) {
            // w^n = w^{n-1} + L d^n; the source enters b (w^n + q) below
            wn[p] = add2(half(din, p), lap[p]);
            lap[p] = wn[p];
        }
        if (inj) lap[p] = add2(lap[p], pk(sqv[j], sqv[j + 1]));
    }
    // the increment the update starts from: d^n (the own column of X in the (w, d) form)
    const P4 &dprev = WD ? cc : din;
    f2 d[2];
    if (interior) {
        d[0] = fma2(bb.a, lap[0], dprev.a);
        d[1] = fma2(bb.b, lap[1], dprev.b);
#pragma unroll
        for (int j = 0; j < 4; j++) sdv[j] = 0.f;
    } else {
        const float sdz = damp_term(z, G.nz, G.nbl, G.hs0z, G.inv_nbl);
        const f2 one = dup(1.f);
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const f2 sd = add2(pk(sdx[2 * p], sdx[2 * p + 1]), dup(sdz));
            const f2 t = fma2(half(bb, p), lap[p], mul2(sub2(one, sd), half(dprev, p)));
            float o0, o1;
            upk(add2(one, sd), o0, o1);
            d[p] = mul2(t, pk(rcp_approx(o0), rcp_approx(o1)));
            upk(sd, sdv[2 * p], sdv[2 * p + 1]);
        }
    }
    if (WD) {
        un.a = d[0];   // X^{n+1} = d^{n+1}
        un.b = d[1];
        dn.a = wn[0];  // Y^{n+1} = w^n
        dn.b = wn[1];
    } else {
        dn.a = d[0];
        dn.b = d[1];
        un.a = add2(cc.a, d[0]);
        un.b = add2(cc.b, d[1]);
    }
}

// Zero the columns at or beyond the row length (the row padding of the internal layout).
__device__ __forceinline__ void zero_pad(int xc, int NX, P4 &dn, P4 &un)
{
    float d[4], u[4];
    upk(dn.a, d[0], d[1]);
    upk(dn.b, d[2], d[3]);
    upk(un.a, u[0], u[1]);
    upk(un.b, u[2], u[3]);
#pragma unroll
    for (int j = 0; j < 4; j++)
        if (xc + j >= NX) d[j] = u[j] = 0.f;
    dn.a = pk(d[0], d[1]);
    dn.b = pk(d[2], d[3]);
    un.a = pk(u[0], u[1]);
    un.b = pk(u[2], u[3]);
}

}  // namespace step
}  // namespace wp
