// Device code of the D3Q27 central-Hermite MRT step (included once per
// storage precision by step_fp64.cu / step_fp32.cu / step_fp16s.cu).
//
// Method (arXiv 2204.10566):
//   f_i(x + c_i, t + 1) = f_i + [T^-1 S T (f^eq - f)]_i           (Sec. 2.1)
//   T_{m,i} = H_m(c_i - u): central Hermite moments                 (Sec. 2.1)
//   f^eq: full Hermite expansion on D3Q27 (Appendix A), whose central
//   moments are (rho, 0, ..., 0)                                    (Appendix A)
//   second-order moments relaxed at omega, orders 3..6 at the ghost rates
//   (default 1, Appendix A).
//
// GB300 design: pull scheme over a fluid-only slot layout (rows of cells
// contiguous along the lattice's longer axis), structure-of-arrays
// populations stored as deviations from the lattice weights; one warp per
// tile of up to 32 cells of a row (FP32) or one thread per cell (FP16S,
// FP64), with the inlet/outlet nodes and the interpolated-wall cells in
// kernels of their own on a second stream.  Every pull source has a
// slot (wall links read a ghost slot the cell filled with its reflected
// population in the previous step), so the gather is 27 unconditional
// coalesced loads at nb[j] + x - cx.  Because T(u) is the tensor product of
// three 1-D 3x3 transforms, T and its inverse are applied as a cascade of
// 1-D passes in registers; with the default ghost rates only the six
// second-order central moments survive relaxation and the inverse is the
// product-form equilibrium plus six correction terms.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "lbm_internal.h"

// Minimum resident blocks per SM requested for the FP32 / FP16S step kernel
// (caps its registers: 65536 / (threads * blocks)); FP64 is left uncapped.
#ifndef LBM_STEP_MIN_BLOCKS
#define LBM_STEP_MIN_BLOCKS 8
#endif
// The same for the kernel of the cells with interpolated walls, which keeps
// the wall record and the own-slot values of a cell in registers as well.
// When the FP32 chunk kernel runs (LBM_FLUID_KERNEL=chunk), the inlet/outlet
// nodes ride in its trailing blocks instead of a launch of their own: +2 % on
// the Re 3500 nozzle, although the node path spills at the fluid path's
// register cap.  In FP16S the fused kernel spilled in the fluid path too, and
// FP64's uncapped fluid path would lose occupancy, so both keep the separate
// launch.
// FP16S: gather and own-slot stores addressed from one pointer per line
// (the three values of a line sit at +1, +stride, +2 stride - 1 from it):
// +4 % / +7 % on the Re 3500 / Re 6500 nozzles, while FP32 lost 4 %, so FP32
// keeps per-population offsets.
#ifndef LBM_LINE_POINTERS
#define LBM_LINE_POINTERS 1
#endif
#ifndef LBM_FUSE_BOUNDARY
#define LBM_FUSE_BOUNDARY 1
#endif
// Warp-uniform fast path of the FP32 / FP16S fluid kernel for warps of fluid
// cells without wall links (fluid_lane_voted); 0 runs every warp through the
// general line sink.
#ifndef LBM_FAST_PATH
#define LBM_FAST_PATH 1
#endif
#ifndef LBM_STEP_MIN_BLOCKS_WALLQ
#define LBM_STEP_MIN_BLOCKS_WALLQ 4
#endif
// L2 prefetch lookahead of the fluid kernel, in percent of the blocks
// resident on the device (0 disables the prefetch).  At 8 blocks per SM the
// FP32 kernel keeps enough loads in flight on its own (the prefetch measured
// neutral, +60 MB of DRAM reads per Re 3500 step), and FP16S runs 2-3 %
// slower with it; both default to off.
#ifndef LBM_PREFETCH_AHEAD_PCT
#define LBM_PREFETCH_AHEAD_PCT 0
#endif
#ifndef LBM_PREFETCH_AHEAD_PCT_FP16S
#define LBM_PREFETCH_AHEAD_PCT_FP16S 0
#endif


namespace lbm {

// ------------------------------------------------------------- storage types

template <int P>
struct Storage;

template <>
struct Storage<0> {  // FP64 deviations
    using T = double;
    using R = double;
    static __device__ __forceinline__ R load(const T *p, R) { return __ldg(p); }
    static __device__ __forceinline__ R load_raw(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void store_raw(T *p, R v) { *p = v; }
    static constexpr bool SCALED = false;
    static __device__ __forceinline__ void store(T *p, R v, R) { *p = v; }
};

template <>
struct Storage<1> {  // FP32 deviations
    using T = float;
    using R = float;
    static __device__ __forceinline__ R load(const T *p, R) { return __ldg(p); }
    static __device__ __forceinline__ R load_raw(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void store_raw(T *p, R v) { *p = v; }
    static constexpr bool SCALED = false;
    static __device__ __forceinline__ void store(T *p, R v, R) { *p = v; }
};

template <>
struct Storage<2> {  // FP16 (f - w) * s, FP32 arithmetic
    using T = __half;
    using R = float;
    static __device__ __forceinline__ R load(const T *p, R inv_s) { return __half2float(__ldg(p)) * inv_s; }
    static __device__ __forceinline__ R load_raw(const T *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void store_raw(T *p, R v) { *p = __float2half_rn(v); }
    static constexpr bool SCALED = true;
    static __device__ __forceinline__ void store(T *p, R v, R s) { *p = __float2half_rn(v * s); }
};

// ----------------------------------------------------------------- stencil

__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i) { return i / 9 - 1; }

// Storage addressing of a lattice whose rows run along axis AX (0: x, 2: z):
// the pull source of population i of the cell at row position p is slot
// nb[row_line<AX>(i)] + p - c_row<AX>(i).
template <int AX>
__host__ __device__ constexpr int c_row(int i) { return AX == 0 ? cx_of(i) : cz_of(i); }
template <int AX>
__host__ __device__ constexpr int row_line(int i) { return AX == 0 ? i / 3 : (cx_of(i) + 1) + 3 * (cy_of(i) + 1); }
// Population of storage line j with c_row = k - 1 (k = 0, 1, 2).
template <int AX>
__host__ __device__ constexpr int line_pop(int j, int k) { return AX == 0 ? 3 * j + k : j + 9 * k; }

// 1-D Gauss-Hermite weights of the third-order quadrature (Appendix A).
// Scalar type of R (F2 holds two FP32 values).
template <class R>
struct ScalarOf {
    using type = R;
};
template <>
struct ScalarOf<struct F2> {
    using type = float;
};

template <class R>
__device__ __forceinline__ R w1(int c) {
    using X = typename ScalarOf<R>::type;
    return R(c == 0 ? X(2) / X(3) : X(1) / X(6));
}

template <class R>
__device__ __forceinline__ R theta0() {
    using X = typename ScalarOf<R>::type;
    return R(X(1) / X(3));
}

// The rational constant a / b in the scalar precision of R.
template <class R>
__device__ __forceinline__ R cst(int a, int b) {
    using X = typename ScalarOf<R>::type;
    return R(X(a) / X(b));
}

// 1-D inverse-transform columns at velocity u (T_1D(u)^-1, column k = g_k):
//   g0(c) = w(c) + d(c), d(0) = -u^2, d(+-1) = (u^2 +- u)/2
//   g1(0) = -2u, g1(+-1) = u +- 1/2;  g2(0) = -1, g2(+-1) = 1/2.
// g0 is also the 1-D factor of the product-form equilibrium.
template <class R>
struct Axis {
    R d[3], g0[3], g1[3];
    __device__ __forceinline__ explicit Axis(R u) {
        const R u2 = u * u, h = R(0.5);
        d[0] = h * (u2 - u);
        d[1] = -u2;
        d[2] = h * (u2 + u);
        g0[0] = w1<R>(-1) + d[0];
        g0[1] = w1<R>(0) + d[1];
        g0[2] = w1<R>(1) + d[2];
        g1[0] = u - h;
        g1[1] = R(-2) * u;
        g1[2] = u + h;
    }
};

template <class R>
__device__ __forceinline__ R g2(int c) { return c == 0 ? R(-1) : R(0.5); }

// Equilibrium deviation f^eq_i(rho, u) - w_i in product form, written so
// that no O(1) cancellation occurs:
//   rho prod(w + d) - prod w = (rho - 1) w_i + rho (dx gy gz + wx (dy gz + wy dz)).
template <class R>
__device__ __forceinline__ void eq_deviation(R rho, const Axis<R> &X, const Axis<R> &Y, const Axis<R> &Z,
                                             R (&out)[27]) {
    const R drho = rho - R(1);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int cy = j % 3 - 1, cz = j / 3 - 1;
        const R wy = w1<R>(cy), wz = w1<R>(cz);
        const R E = Y.g0[cy + 1] * Z.g0[cz + 1];
        const R D = Y.d[cy + 1] * Z.g0[cz + 1] + wy * Z.d[cz + 1];
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx) {
            const R wx = w1<R>(cx);
            out[3 * j + cx + 1] = drho * (wx * wy * wz) + rho * (X.d[cx + 1] * E + wx * D);
        }
    }
}

// d_i += f^eq_i(rho_b, u_b) - f^eq_i(rho_f, u_f), line by line so that only
// a few values are live besides d (keeps the boundary path from raising the
// register count of the whole kernel).
template <class R>
__device__ __forceinline__ void add_eq_difference(R rb, R uxb, R uyb, R uzb, R rf, R uxf, R uyf, R uzf,
                                                  R (&d)[27]) {
    const Axis<R> Xb(uxb), Yb(uyb), Zb(uzb), Xf(uxf), Yf(uyf), Zf(uzf);
    const R db = rb - R(1), df = rf - R(1);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int cy = j % 3 - 1, cz = j / 3 - 1;
        const R wy = w1<R>(cy), wz = w1<R>(cz);
        const R Eb = Yb.g0[cy + 1] * Zb.g0[cz + 1], Ef = Yf.g0[cy + 1] * Zf.g0[cz + 1];
        const R Db = Yb.d[cy + 1] * Zb.g0[cz + 1] + wy * Zb.d[cz + 1];
        const R Df = Yf.d[cy + 1] * Zf.g0[cz + 1] + wy * Zf.d[cz + 1];
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx) {
            const R w = w1<R>(cx) * wy * wz;
            d[3 * j + cx + 1] += (db * w + rb * (Xb.d[cx + 1] * Eb + w1<R>(cx) * Db)) -
                                 (df * w + rf * (Xf.d[cx + 1] * Ef + w1<R>(cx) * Df));
        }
    }
}

// ------------------------------------------------------ viscous stress

// Viscous stress of a cell from its pre-collision second-order central
// Hermite moments a_ab = sum_i ((c - u)_a (c - u)_b - theta0 delta_ab) f_i
// (Appendix A strain-rate relation, with the sign of the non-equilibrium
// stress): sigma_ab = 2 rho nu S_ab = -(1 - omega/2) a_ab, accumulated in
// FP64 on statistics sample steps (Sec. 2.2 viscous shear stress).
template <class R>
__device__ __forceinline__ void record_stress(const StepArgs &a, int slot, R omega, const R (&a2)[6]) {
    if ((a.flags & (STEP_STATS | STEP_STATS_FULL)) != (STEP_STATS | STEP_STATS_FULL)) return;
    const double f = -(1.0 - 0.5 * (double)omega);
    double *p = a.stats + 11 * (int64_t)a.stride + slot;
#pragma unroll
    for (int q = 0; q < 6; ++q) p[q * a.stride] += f * (double)a2[q];
}

// --------------------------------------------------------------- collision

__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Packed FP32 (two values per instruction, sm_100 and later) for the inverse
// transform of the rate-1 collision.  Off: -DLBM_PACKED_F32=0.
#ifndef LBM_PACKED_F32
#define LBM_PACKED_F32 1
#endif

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// Two cells' FP32 values on the packed pipe: every arithmetic operation of
// the collision applies to both lanes with one instruction.
struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ explicit F2(float2 w) : v(w) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, bc2(-1.0f), a.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2 &operator*=(F2 &a, F2 b) { return a = a * b; }
__device__ __forceinline__ F2 recip(F2 x) { return F2(make_float2(__frcp_rn(x.v.x), __frcp_rn(x.v.y))); }

// Shared inputs of the per-line inverse (see collide_ghost1).
struct PairCoef {
    float Axx, Ayy, Azz, Axy, Axz, Ayz, rho_o, drho_o, ux, ux2h, uxh;
};

// One line (cy, cz) of the inverse: f*_i - w_i for cx = -1, 0, +1.
template <class R, int J, class Out>
__device__ __forceinline__ void inverse_line(R Axx, R Ayy, R Azz, R Axy, R Axz, R Ayz, R rho_o, R drho_o, R ux, R ux2h,
                                             R uxh, const Axis<R> &Y, const Axis<R> &Z, const Out &sink) {
    constexpr int cy = J % 3 - 1, cz = J / 3 - 1;
    const R h = R(0.5);
    const R wy = w1<R>(cy);
    const R gy0 = Y.g0[cy + 1], gz0 = Z.g0[cz + 1], gy1 = Y.g1[cy + 1], gz1 = Z.g1[cz + 1];
    const R E = gy0 * gz0;
    const R D = Y.d[cy + 1] * gz0 + wy * Z.d[cz + 1];
    const R C0 = Ayy * g2<R>(cy) * gz0 + Azz * gy0 * g2<R>(cz) + Ayz * gy1 * gz1;
    const R B1 = Axy * gy1 * gz0 + Axz * gy0 * gz1;
    const R B2 = Axx * E;
    const R Bw = drho_o * (wy * w1<R>(cz)) + rho_o * D + C0;
    const R Bd = rho_o * E + C0;
    const R v0 = cst<R>(2, 3) * Bw - R(2) * (ux2h * Bd + ux * B1) - B2;
    const R S = cst<R>(1, 6) * Bw + ux2h * Bd + ux * B1 + h * B2;
    const R A = uxh * Bd + h * B1;
    sink(J, S - A, v0, S + A);
}

// Two lines of the inverse at once.  The pair differs along one axis ("v",
// c = -1 in .x and +1 in .y) and shares the other ("f"); the line formulas
// are symmetric in y and z once the diagonal and mixed second-order
// coefficients are relabelled, so one routine serves both kinds of pair:
//   E = g0v g0f,  D = dv g0f + (1/6) df,
//   C0 = Avv (1/2) g0f + Aff g2f g0v + Ayz g1f g1v,
//   B1 = Axv g0f g1v + Axf g1f g0v,  B2 = Axx E,
// with the same Bw, Bd, v0, S, A as the scalar line.
template <int JA, int JB, class Out>
__device__ __forceinline__ void inverse_pair(const PairCoef &c, const Axis<float> &Y, const Axis<float> &Z,
                                             const Out &sink) {
    constexpr bool YV = (JA / 3) == (JB / 3);  // same cz: y varies
    constexpr int cf = YV ? JA / 3 - 1 : JA % 3 - 1;  // fixed axis velocity
    const Axis<float> &V = YV ? Y : Z;
    const Axis<float> &F = YV ? Z : Y;
    const float Avv = YV ? c.Ayy : c.Azz, Aff = YV ? c.Azz : c.Ayy;
    const float Axv = YV ? c.Axy : c.Axz, Axf = YV ? c.Axz : c.Axy;
    const float f0 = F.g0[cf + 1], f1 = F.g1[cf + 1], fd = F.d[cf + 1], fw = w1<float>(cf), fg2 = g2<float>(cf);
    const float2 v0_ = make_float2(V.g0[0], V.g0[2]), v1_ = make_float2(V.g1[0], V.g1[2]);
    const float2 vd = make_float2(V.d[0], V.d[2]);
    const float2 E = __fmul2_rn(v0_, bc2(f0));
    const float2 D = __ffma2_rn(vd, bc2(f0), bc2(fd * (1.0f / 6.0f)));
    const float2 C0 = __ffma2_rn(v1_, bc2(c.Ayz * f1), __ffma2_rn(v0_, bc2(Aff * fg2), bc2(0.5f * Avv * f0)));
    const float2 hB1 = __ffma2_rn(v1_, bc2(0.5f * Axv * f0), __fmul2_rn(v0_, bc2(0.5f * Axf * f1)));
    const float2 nB2 = __fmul2_rn(v0_, bc2(-c.Axx * f0));
    const float2 hB2 = __fmul2_rn(v0_, bc2(0.5f * c.Axx * f0));
    const float2 Bw = __ffma2_rn(bc2(c.rho_o), D, __fadd2_rn(C0, bc2(c.drho_o * (fw * (1.0f / 6.0f)))));
    const float2 Bd = __ffma2_rn(bc2(c.rho_o), E, C0);
    const float2 t = __ffma2_rn(bc2(c.ux2h), Bd, __fmul2_rn(bc2(2.0f * c.ux), hB1));
    const float2 o0 = __ffma2_rn(bc2(2.0f / 3.0f), Bw, __ffma2_rn(bc2(-2.0f), t, nB2));
    const float2 S = __ffma2_rn(bc2(1.0f / 6.0f), Bw, __fadd2_rn(t, hB2));
    const float2 A = __ffma2_rn(bc2(c.uxh), Bd, hB1);
    const float2 om = __ffma2_rn(bc2(-1.0f), A, S), op = __fadd2_rn(S, A);
    sink(JA, om.x, o0.x, op.x);
    sink(JB, om.y, o0.y, op.y);
}

// Writes a line of three outputs (cx = -1, 0, +1 of line j) back into d.
template <class R>
struct ToArray {
    R (&d)[27];
    __device__ __forceinline__ void moments(R, const R (&)[6]) const {}
    __device__ __forceinline__ void operator()(int j, R vm, R v0, R vp) const {
        d[3 * j] = vm;
        d[3 * j + 1] = v0;
        d[3 * j + 2] = vp;
    }
};

// ToArray that also records the viscous stress of the cell at `slot`.
template <class R>
struct ToArrayStress {
    const StepArgs &a;
    int slot;
    R (&d)[27];
    __device__ __forceinline__ void moments(R omega, const R (&a2)[6]) const { record_stress(a, slot, omega, a2); }
    __device__ __forceinline__ void operator()(int j, R vm, R v0, R vp) const { ToArray<R>{d}(j, vm, v0, vp); }
};

// Identity conversion of a collision input.
struct SameInput {
    template <class R>
    __device__ __forceinline__ R operator()(R v) const { return v; }
};

// Moment sums of the default-rate collision from its 27 inputs (cvt turns an
// input into R): m = drho, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz, the
// sums of (f - w) weighted by 1, c, and c_a c_b.  The x-pass sums each
// (cy, cz) line with weights 1, cx, cx^2; the other axes follow.
template <class R, class In, class Cvt>
__device__ __forceinline__ void ghost1_sums(const In (&d)[27], const Cvt &cvt, R (&m)[10]) {
    R s0[9], s1[9], s2[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const R a = cvt(d[3 * j]), b = cvt(d[3 * j + 1]), c = cvt(d[3 * j + 2]);
        s0[j] = (a + b) + c;
        s1[j] = c - a;
        s2[j] = c + a;
    }
    R drho = 0, jx = 0, jy = 0, jz = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pxz = 0, pyz = 0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int cy = j % 3 - 1, cz = j / 3 - 1;
        drho += s0[j];
        jx += s1[j];
        pxx += s2[j];
        if (cy != 0) {
            jy += cy > 0 ? s0[j] : -s0[j];
            pyy += s0[j];
            pxy += cy > 0 ? s1[j] : -s1[j];
        }
        if (cz != 0) {
            jz += cz > 0 ? s0[j] : -s0[j];
            pzz += s0[j];
            pxz += cz > 0 ? s1[j] : -s1[j];
        }
        if (cy != 0 && cz != 0) pyz += (cy * cz) > 0 ? s0[j] : -s0[j];
    }
    m[0] = drho, m[1] = jx, m[2] = jy, m[3] = jz, m[4] = pxx;
    m[5] = pyy, m[6] = pzz, m[7] = pxy, m[8] = pxz, m[9] = pyz;
}

// The rest of the default-rate collision from the moment sums: rho, u, the
// six second-order central Hermite moments, their relaxation, and the
// inverse transform, line by line into sink(j, f*_{3j} - w, f*_{3j+1} - w,
// f*_{3j+2} - w).  With SCALED the sums are of (f - w) / in_scale and the
// outputs are (f* - w) * out_scale: the scales act on the ten moments and
// the eight output coefficients instead of on the 54 populations.
template <class R, bool SCALED, class Out>
__device__ __forceinline__ void ghost1_finish(const R (&m)[10], R omega, R &rho, R &ux, R &uy, R &uz, R in_scale,
                                              R out_scale, const Out &sink) {
    R drho = m[0], jx = m[1], jy = m[2], jz = m[3], pxx = m[4], pyy = m[5], pzz = m[6], pxy = m[7], pxz = m[8],
      pyz = m[9];
    if constexpr (SCALED) {
        drho *= in_scale;
        jx *= in_scale;
        jy *= in_scale;
        jz *= in_scale;
        pxx *= in_scale;
        pyy *= in_scale;
        pzz *= in_scale;
        pxy *= in_scale;
        pxz *= in_scale;
        pyz *= in_scale;
    }
    rho = R(1) + drho;
    const R inv = recip(rho);
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
    // Second-order central Hermite moments sum_i ((c-u)_a (c-u)_b - theta0 delta_ab) f_i,
    // from the deviation moments (sum c_a c_b w = theta0 delta_ab).
    const R th = theta0<R>();
    const R k = SCALED ? (R(1) - omega) * out_scale : R(1) - omega;
    const R rho_o = SCALED ? rho * out_scale : rho, drho_o = SCALED ? drho * out_scale : drho;
    const R a2[6] = {pxx - rho * ux * ux - th * drho, pyy - rho * uy * uy - th * drho, pzz - rho * uz * uz - th * drho,
                     pxy - rho * ux * uy,            pxz - rho * ux * uz,            pyz - rho * uy * uz};
    sink.moments(omega, a2);
    const R Axx = k * a2[0];
    const R Ayy = k * a2[1];
    const R Azz = k * a2[2];
    const R Axy = k * a2[3];
    const R Axz = k * a2[4];
    const R Ayz = k * a2[5];
    // Inverse: f* = rho prod g0 + sum over the six relaxed second-order moments
    // of A_m prod_a g_{m_a}; orders 1 and 3..6 are zero after relaxation.
    // Per (cy, cz) line the x-dependence is spanned by {w, d, g1, g2}(cx):
    //   f*_i - w_i = wx Bw + dx Bd + g1x B1 + g2x B2,
    // and for cx = +-1 this splits into S +- A.
    const Axis<R> Y(uy), Z(uz);
    const R h = R(0.5);
    const R ux2h = h * ux * ux, uxh = h * ux;
#if LBM_PACKED_F32
    if constexpr (std::is_same<R, float>::value) {
        // Lines in pairs on the packed FP32 pipe (two lanes per instruction):
        // (cy = -1, +1) at each cz, then (cz = -1, +1) at cy = 0; line 4 alone.
        const PairCoef c{Axx, Ayy, Azz, Axy, Axz, Ayz, rho_o, drho_o, ux, ux2h, uxh};
        inverse_pair<0, 2>(c, Y, Z, sink);
        inverse_pair<3, 5>(c, Y, Z, sink);
        inverse_pair<6, 8>(c, Y, Z, sink);
        inverse_pair<1, 7>(c, Y, Z, sink);
        inverse_line<R, 4>(Axx, Ayy, Azz, Axy, Axz, Ayz, rho_o, drho_o, ux, ux2h, uxh, Y, Z, sink);
        return;
    }
#endif
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int cy = j % 3 - 1, cz = j / 3 - 1;
        const R wy = w1<R>(cy);
        const R gy0 = Y.g0[cy + 1], gz0 = Z.g0[cz + 1], gy1 = Y.g1[cy + 1], gz1 = Z.g1[cz + 1];
        const R E = gy0 * gz0;
        const R D = Y.d[cy + 1] * gz0 + wy * Z.d[cz + 1];
        const R C0 = Ayy * g2<R>(cy) * gz0 + Azz * gy0 * g2<R>(cz) + Ayz * gy1 * gz1;
        const R B1 = Axy * gy1 * gz0 + Axz * gy0 * gz1;
        const R B2 = Axx * E;
        const R Bw = drho_o * (wy * w1<R>(cz)) + rho_o * D + C0;
        const R Bd = rho_o * E + C0;
        // cx = 0: w = 2/3, d = -ux^2, g1 = -2 ux, g2 = -1
        const R v0 = cst<R>(2, 3) * Bw - R(2) * (ux2h * Bd + ux * B1) - B2;
        // cx = +-1: w = 1/6, d = (ux^2 +- ux)/2, g1 = ux +- 1/2, g2 = 1/2
        const R S = cst<R>(1, 6) * Bw + ux2h * Bd + ux * B1 + h * B2;
        const R A = uxh * Bd + h * B1;
        sink(j, S - A, v0, S + A);  // the line's outputs leave registers at once
    }
}

// Collision with the default ghost rates (all 1).  d holds f_i - w_i on entry;
// the post-collision f*_i - w_i go to the sink line by line, or back into d
// without one.  rho, u receive the (conserved) moments.  With SCALED, d holds
// (f_i - w_i) / in_scale and the outputs are (f*_i - w_i) * out_scale.
template <class R, bool SCALED = false, class Out = ToArray<R>>
__device__ __forceinline__ void collide_ghost1(R (&d)[27], R omega, R &rho, R &ux, R &uy, R &uz,
                                               R in_scale = R(1), R out_scale = R(1), const Out *sink = nullptr) {
    R m[10];
    ghost1_sums(d, SameInput{}, m);
    if (sink)
        ghost1_finish<R, SCALED>(m, omega, rho, ux, uy, uz, in_scale, out_scale, *sink);
    else
        ghost1_finish<R, SCALED>(m, omega, rho, ux, uy, uz, in_scale, out_scale, ToArray<R>{d});
}

// 1-D forward central Hermite factor h_k(c - u): 1, c - u, (c - u)^2 - theta0.
template <class R>
__device__ __forceinline__ R hfwd(int k, int c, R u) {
    const R x = R(c) - u;
    return k == 0 ? R(1) : (k == 1 ? x : x * x - theta0<R>());
}

// Collision with general ghost rates: the full 27-moment cascade.
//   dA = T(u) (f - w), A = e(u) + dA with e_m = prod_a e_{m_a}(u_a),
//   e0 = 1, e1 = -u, e2 = u^2 (the central moments of the weights);
//   A* = A + S (A^eq - A), A^eq = (rho, 0, ..., 0);
//   f* - w = T^-1 (A* - e).
template <class R, class Sink = ToArray<R>>
__device__ __forceinline__ void collide_general(R (&d)[27], R omega, const R (&ghost)[4], R &rho, R &ux,
                                                R &uy, R &uz, const Sink *sink = nullptr) {
    R drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        drho += d[i];
        if (cx_of(i)) jx += cx_of(i) > 0 ? d[i] : -d[i];
        if (cy_of(i)) jy += cy_of(i) > 0 ? d[i] : -d[i];
        if (cz_of(i)) jz += cz_of(i) > 0 ? d[i] : -d[i];
    }
    rho = R(1) + drho;
    const R inv = recip(rho);
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
    const R u[3] = {ux, uy, uz};
    // forward cascade, axis by axis; index layout a[kx + 3 ky + 9 kz] after all passes
    R a[27];
#pragma unroll
    for (int j = 0; j < 9; ++j)  // x-pass over lines (cy, cz)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            a[3 * j + k] = hfwd<R>(k, -1, ux) * d[3 * j] + hfwd<R>(k, 0, ux) * d[3 * j + 1] +
                           hfwd<R>(k, 1, ux) * d[3 * j + 2];
    R b[27];
#pragma unroll
    for (int kx = 0; kx < 3; ++kx)  // y-pass
#pragma unroll
        for (int cz = 0; cz < 3; ++cz)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                b[kx + 3 * k + 9 * cz] = hfwd<R>(k, -1, uy) * a[kx + 9 * cz] + hfwd<R>(k, 0, uy) * a[kx + 3 + 9 * cz] +
                                         hfwd<R>(k, 1, uy) * a[kx + 6 + 9 * cz];
#pragma unroll
    for (int kx = 0; kx < 3; ++kx)  // z-pass
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                a[kx + 3 * ky + 9 * k] = hfwd<R>(k, -1, uz) * b[kx + 3 * ky] + hfwd<R>(k, 0, uz) * b[kx + 3 * ky + 9] +
                                         hfwd<R>(k, 1, uz) * b[kx + 3 * ky + 18];
    if (sink) {  // second-order central Hermite moments A_m = e_m + a_m
        const R a2[6] = {ux * ux + a[2], uy * uy + a[6], uz * uz + a[18],
                         ux * uy + a[4], ux * uz + a[10], uy * uz + a[12]};
        sink->moments(omega, a2);
    }
    // relax; work with D_m = A*_m - e_m
#pragma unroll
    for (int m = 0; m < 27; ++m) {
        const int kx = m % 3, ky = (m / 3) % 3, kz = m / 9, n = kx + ky + kz;
        R e = R(1);
        const int ks[3] = {kx, ky, kz};
#pragma unroll
        for (int q = 0; q < 3; ++q) e *= ks[q] == 0 ? R(1) : (ks[q] == 1 ? -u[q] : u[q] * u[q]);
        if (n == 0) {
            a[m] = drho;  // A*_0 = rho, e_0 = 1
        } else if (n == 1) {
            a[m] = -e;    // A*_1 = 0
        } else {
            const R rate = n == 2 ? omega : ghost[n - 3];
            a[m] = (R(1) - rate) * (e + a[m]) - e;  // A* - e with A^eq_m = 0
        }
    }
    // inverse cascade: z, then y, then x
    const Axis<R> X(ux), Y(uy), Z(uz);
#pragma unroll
    for (int kx = 0; kx < 3; ++kx)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int cz = -1; cz <= 1; ++cz)
                b[kx + 3 * ky + 9 * (cz + 1)] = Z.g0[cz + 1] * a[kx + 3 * ky] + Z.g1[cz + 1] * a[kx + 3 * ky + 9] +
                                                g2<R>(cz) * a[kx + 3 * ky + 18];
#pragma unroll
    for (int kx = 0; kx < 3; ++kx)
#pragma unroll
        for (int cz = 0; cz < 3; ++cz)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
                a[kx + 3 * (cy + 1) + 9 * cz] = Y.g0[cy + 1] * b[kx + 9 * cz] + Y.g1[cy + 1] * b[kx + 3 + 9 * cz] +
                                                g2<R>(cy) * b[kx + 6 + 9 * cz];
#pragma unroll
    for (int j = 0; j < 9; ++j)
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx)
            d[3 * j + cx + 1] = X.g0[cx + 1] * a[3 * j] + X.g1[cx + 1] * a[3 * j + 1] + g2<R>(cx) * a[3 * j + 2];
}

// ---------------------------------------------------------------- streaming

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// The nine neighbour-row bases of a row record (j = (cy+1) + 3 (cz+1)).
__device__ __forceinline__ void load_row(const int4 *row_nb, int row, int (&nb)[9]) {
    const int4 a = __ldg(row_nb + 3 * row), b = __ldg(row_nb + 3 * row + 1), c = __ldg(row_nb + 3 * row + 2);
    nb[0] = a.x; nb[1] = a.y; nb[2] = a.z; nb[3] = a.w;
    nb[4] = b.x; nb[5] = b.y; nb[6] = b.z; nb[7] = b.w;
    nb[8] = c.x;
}

// Element offset of (population i, slot s): i * stride + s, in 32-bit
// unsigned arithmetic when the buffer allows (see MAX_SLOTS_32).
template <bool WIDE>
__device__ __forceinline__ typename std::conditional<WIDE, int64_t, uint32_t>::type
elem(int i, int64_t stride, int s) {
    if constexpr (WIDE)
        return (int64_t)i * stride + s;
    else
        return (uint32_t)i * (uint32_t)stride + (uint32_t)s;
}

// Pull gather of the cell at x in the row with bases nb: d_i = f*_i(x - c_i)
// from slot nb[j] + x - cx of population array i.  For a wall link that slot
// is the ghost slot holding f*_{26-i}(x) (halfway bounce-back, i.e.
// Bouzidi's interpolated bounce-back at q = 1/2, Sec. 2.2).
template <int P, bool WIDE, int AX, bool RAW = false>
__device__ __forceinline__ void gather(const StepArgs &a, const int (&nb)[9], int x, typename Storage<P>::R (&d)[27]) {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    const T *fin = static_cast<const T *>(a.fin);
    const R inv_s = R(a.inv_scale);
#if LBM_LINE_POINTERS
    if constexpr (!WIDE && P == 2) {
        // one pointer per storage line j (its three populations pull from
        // row nb[j]); the pulls sit at +1, +(k1 - k0) stride, +(k2 - k0) stride - 1
        const uint32_t st = (uint32_t)a.stride;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            constexpr int dk = line_pop<AX>(0, 1) - line_pop<AX>(0, 0);
            const T *pj = fin + ((uint32_t)line_pop<AX>(j, 0) * st + (uint32_t)(nb[j] + x));
            const T *q[3] = {pj + 1, pj + dk * st, pj + 2 * dk * st - 1};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int i = line_pop<AX>(j, k);
                d[i] = RAW ? S::load_raw(q[k]) : S::load(q[k], inv_s);
            }
        }
        return;
    }
#endif
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const T *p = fin + elem<WIDE>(i, a.stride, nb[row_line<AX>(i)] + x - c_row<AX>(i));
        d[i] = RAW ? S::load_raw(p) : S::load(p, inv_s);  // RAW: storage value, scale applied later
    }
}

// Bouzidi's interpolated bounce-back (Sec. 2.2) on the wall links of a cell
// whose wall distances were given (lbm_set_wall_q).  The gather has already
// put f*_ib(x) into d[i] for every wall link i (the ghost slot, halfway
// bounce-back; ib = 26 - i is the direction from x towards the wall), and the
// pull of ib into d[ib].  With q the wall's distance from x as a fraction of
// the link:
//   q <  1/2: f_i = 2q f*_ib(x) + (1 - 2q) f*_ib(x + c_i)   (= d[ib], unless
//             x + c_i is a wall too: then the halfway value stays),
//   q >= 1/2: f_i = f*_ib(x) / (2q) + (1 - 1/(2q)) f*_i(x)   (own slot, array i).
// Every term is a deviation (or scaled deviation) from w_i = w_ib, and the
// coefficients sum to 1, so the storage form needs no conversion.
template <int P, bool WIDE, bool RAW>
__device__ __forceinline__ void interpolate_walls(const StepArgs &a, int k, int slot, uint32_t links,
                                                  typename Storage<P>::R (&d)[27]) {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    if (k < 0) return;
    // the record as two 16-byte loads; byte i = q of link i in 1/256
    const uint4 *rec = reinterpret_cast<const uint4 *>(a.wall_q) + 2 * (size_t)k;
    const uint4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
    const uint32_t w[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    const T *fin = static_cast<const T *>(a.fin);
    // own-slot values for the links with q > 1/2, all loads issued first
    R own[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const uint32_t q8 = (w[i >> 2] >> (8 * (i & 3))) & 0xFFu;
        own[i] = R(0);
        if ((links & (1u << i)) && q8 > 128u) {
            const T *p = fin + elem<WIDE>(i, a.stride, slot);
            own[i] = RAW ? S::load_raw(p) : S::load(p, R(a.inv_scale));
        }
    }
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        if (!(links & (1u << i))) continue;
        const uint32_t q8 = (w[i >> 2] >> (8 * (i & 3))) & 0xFFu;
        const int ib = 26 - i;
        if (q8 < 128u) {
            if (links & (1u << ib)) continue;
            const R q2 = R(q8) * R(1.0 / 128.0);  // 2q
            d[i] = q2 * d[i] + (R(1) - q2) * d[ib];
        } else if (q8 > 128u) {
            const R c = R(128) / R(q8);  // 1 / (2q)
            d[i] = c * d[i] + (R(1) - c) * own[i];
        }
    }
}

// ------------------------------------------------------------------- inlet

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    // SplitMix64 output function (Steele, Lea and Flood 2014).
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Counter-based uniform variate in [-1, 1) for (seed, step, node, component);
// 24 random bits, exact in binary32.
template <class R>
__device__ __forceinline__ R inlet_noise(uint64_t seed, int64_t step, int64_t node, int comp) {
    uint64_t h = splitmix64(seed);
    h = splitmix64((uint64_t)step + h);
    h = splitmix64((((uint64_t)node << 2) | (uint64_t)comp) + h);
    return R((uint32_t)(h >> 40)) * R(1.0 / 8388608.0) - R(1);
}

// -------------------------------------------------------- block reduction

__device__ __forceinline__ void block_reduce_write(double (&v)[6], double *partials) {
    __shared__ double sh[32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double t = __shfl_down_sync(0xffffffffu, v[k], o);
            v[k] = (k == 4) ? fmax(v[k], t) : v[k] + t;
        }
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = sh[0][k];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
            for (int k = 0; k < 6; ++k) r[k] = (k == 4) ? fmax(r[k], sh[w][k]) : r[k] + sh[w][k];
        double *p = partials + (size_t)blockIdx.x * REDUCE_SLOTS;
#pragma unroll
        for (int k = 0; k < 6; ++k) p[k] = r[k];
    }
}

__device__ __forceinline__ void health_values(double rho, double ux, double uy, double uz, double (&v)[6]) {
    const bool finite = isfinite(rho) && isfinite(ux) && isfinite(uy) && isfinite(uz);
    v[0] = rho;
    v[1] = rho * ux;
    v[2] = rho * uy;
    v[3] = rho * uz;
    v[4] = finite ? sqrt(ux * ux + uy * uy + uz * uz) : 0.0;
    v[5] = finite ? 0.0 : 1.0;
}

// --------------------------------------------------------------- step kernel

template <class R>
__device__ __forceinline__ const FlowParams<R> &flow(const StepArgs &a);
template <>
__device__ __forceinline__ const FlowParams<double> &flow<double>(const StepArgs &a) { return a.pd; }
template <>
__device__ __forceinline__ const FlowParams<float> &flow<float>(const StepArgs &a) { return a.pf; }

// Collision of d in place; the viscous stress is recorded at stress_slot.
template <int P, bool GHOST1>
__device__ __forceinline__ void collide(typename Storage<P>::R (&d)[27], const FlowParams<typename Storage<P>::R> &fp,
                                        typename Storage<P>::R &rho, typename Storage<P>::R &ux,
                                        typename Storage<P>::R &uy, typename Storage<P>::R &uz, const StepArgs &a,
                                        int stress_slot) {
    using R = typename Storage<P>::R;
    const ToArrayStress<R> sink{a, stress_slot, d};
    if (GHOST1)
        collide_ghost1<R, false, ToArrayStress<R>>(d, fp.omega, rho, ux, uy, uz, R(1), R(1), &sink);
    else
        collide_general<R, ToArrayStress<R>>(d, fp.omega, fp.ghost, rho, ux, uy, uz, &sink);
}

// Post-collision state of one cell is in d; write it to its own slot, the
// ghost slots of its wall links, and (periodic row axis) its wrap-around
// copies.
template <int P, bool WIDE, int AX, bool RAW = false>
__device__ __forceinline__ void store_cell_state(const StepArgs &a, const int (&nb)[9], int x, int slot, uint32_t links,
                                                 const typename Storage<P>::R (&d)[27]) {
    using S0 = Storage<P>;
    using T = typename S0::T;
    using R = typename S0::R;
    // RAW: d already holds storage values (scale applied by the collision)
    struct S {
        static __device__ __forceinline__ void store(T *p, R v, R sc) {
            if constexpr (RAW)
                S0::store_raw(p, v);
            else
                S0::store(p, v, sc);
        }
    };
    const R s = R(a.scale);
    T *fout = static_cast<T *>(a.fout);
#pragma unroll
    for (int i = 0; i < 27; ++i) S::store(fout + elem<WIDE>(i, a.stride, slot), d[i], s);
    if (links) {  // wall links: the reflected population waits in the ghost slot
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            if (!(links & (7u << (3 * j)))) continue;  // no wall link among populations 3j .. 3j + 2
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int i = 3 * j + c;
                if (links & (1u << i))
                    S::store(fout + elem<WIDE>(i, a.stride, nb[row_line<AX>(i)] + x - c_row<AX>(i)), d[26 - i], s);
            }
        }
    }
    if (a.periodic_row) {  // wrap-around copies read across the periodic faces of the row axis
        if (x == a.n_row - 1) {
#pragma unroll
            for (int i = 0; i < 27; ++i)
                if (c_row<AX>(i) == 1) S::store(fout + elem<WIDE>(i, a.stride, nb[4] - 1), d[i], s);
        }
        if (x == 0) {
#pragma unroll
            for (int i = 0; i < 27; ++i)
                if (c_row<AX>(i) == -1) S::store(fout + elem<WIDE>(i, a.stride, nb[4] + a.n_row), d[i], s);
        }
    }
}

// Output sink of the fluid update: each line of three post-collision values
// (populations 3j .. 3j + 2) goes to the cell's own slots at once, to the
// ghost slots of the wall links they serve (value i feeds link 26 - i), and
// across a periodic face of the row axis.
// own: bit i set = store value i in the cell's own slot; bit 31 = the lane is
// a fluid cell (the other lanes only fill unread arrays, see fluid_cell).
constexpr uint32_t OWN_FLUID = 1u << 31;

template <int P, bool WIDE, bool RAW, int AX>
struct LineStore {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    const StepArgs &a;
    const int (&nb)[9];
    int x, slot;
    uint32_t links, own;
    __device__ __forceinline__ void put(int i, int s, R v) const {
        T *p = static_cast<T *>(a.fout) + elem<WIDE>(i, a.stride, s);
        if constexpr (RAW)
            S::store_raw(p, v);
        else
            S::store(p, v, R(a.scale));
    }
    __device__ __forceinline__ void moments(R omega, const R (&a2)[6]) const {
        if (own & OWN_FLUID) record_stress(a, slot, omega, a2);
    }
    __device__ __forceinline__ void operator()(int j, R vm, R v0, R vp) const {
#if LBM_LINE_POINTERS
        if constexpr (!WIDE && P == 2) {  // the three own-slot stores of line j from one pointer
            const uint32_t st = (uint32_t)a.stride;
            T *pj = static_cast<T *>(a.fout) + ((uint32_t)(3 * j) * st + (uint32_t)slot);
            const R v[3] = {vm, v0, vp};
            T *q[3] = {pj, pj + st, pj + 2 * st};
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (own & (1u << (3 * j + c))) {
                    if constexpr (RAW)
                        S::store_raw(q[c], v[c]);
                    else
                        S::store(q[c], v[c], R(a.scale));
                }
        } else
#endif
        {
            if (own & (1u << (3 * j))) put(3 * j, slot, vm);
            if (own & (2u << (3 * j))) put(3 * j + 1, slot, v0);
            if (own & (4u << (3 * j))) put(3 * j + 2, slot, vp);
        }
        const int jl = 8 - j;  // links 26 - i of this line's values sit in line 8 - j
        if (links & (7u << (3 * jl))) {
            const R v[3] = {vm, v0, vp};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int k = 26 - (3 * j + c);  // wall link k takes value 3j + c
                if (links & (1u << k)) put(k, nb[row_line<AX>(k)] + x - c_row<AX>(k), v[c]);
            }
        }
        if (a.periodic_row && (own & OWN_FLUID)) {  // wrap-around copies across the periodic row faces
            const R v[3] = {vm, v0, vp};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int i = 3 * j + c;
                if (c_row<AX>(i) == 1 && x == a.n_row - 1) put(i, nb[4] - 1, v[c]);
                if (c_row<AX>(i) == -1 && x == 0) put(i, nb[4] + a.n_row, v[c]);
            }
        }
    }
};

// Output sink of the fast path (a warp of fluid cells without wall links):
// the 27 post-collision values go to the cell's own slots only, with no
// predicate.  FP16S addresses each line's three stores from one pointer, FP32
// by per-population offsets, as LineStore does.
template <int P, bool RAW>
struct OwnStore {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    const StepArgs &a;
    int slot;
    __device__ __forceinline__ void put(T *p, R v) const {
        if constexpr (RAW)
            S::store_raw(p, v);
        else
            S::store(p, v, R(a.scale));
    }
    __device__ __forceinline__ void moments(R omega, const R (&a2)[6]) const { record_stress(a, slot, omega, a2); }
    __device__ __forceinline__ void operator()(int j, R vm, R v0, R vp) const {
        T *out = static_cast<T *>(a.fout);
        const uint32_t st = (uint32_t)a.stride;
        if constexpr (LBM_LINE_POINTERS && P == 2) {
            T *pj = out + ((uint32_t)(3 * j) * st + (uint32_t)slot);
            put(pj, vm);
            put(pj + st, v0);
            put(pj + 2 * st, vp);
        } else {
            put(out + elem<false>(3 * j, a.stride, slot), vm);
            put(out + elem<false>(3 * j + 1, a.stride, slot), v0);
            put(out + elem<false>(3 * j + 2, a.stride, slot), vp);
        }
    }
};

template <class R>
__device__ __forceinline__ void record_cell(const StepArgs &a, int slot, R rho, R ux, R uy, R uz, double (&hv)[6]) {
    if (a.flags & STEP_STATS) {
        const double w = (double)uz;
        a.stats[slot] += w;
        a.stats[a.stride + slot] += w * w;
        if (a.flags & STEP_STATS_FULL) {  // time averages of u, u u and rho (Sec. 2.2)
            const double u[3] = {(double)ux, (double)uy, (double)uz};
            const double uu[6] = {u[0] * u[0], u[1] * u[1], u[2] * u[2], u[0] * u[1], u[0] * u[2], u[1] * u[2]};
            double *p = a.stats + 2 * (int64_t)a.stride + slot;
#pragma unroll
            for (int q = 0; q < 3; ++q) p[q * a.stride] += u[q];
#pragma unroll
            for (int q = 0; q < 6; ++q) p[(3 + q) * a.stride] += uu[q];
            p[15 * a.stride] += (double)rho;
        }
    }
    if (a.flags & STEP_REDUCE) health_values(rho, ux, uy, uz, hv);
}

// Update of the fluid cell in lane `lane` of chunk `chunk` (Sec. 2.1
// evolution equation, pull form): gather, collide, store, refill the ghost
// slots of its wall links.  The chunk's other lanes run the same instruction
// stream on whatever their pull slots hold (all inside the buffer and its
// margins) and store the result only into the arrays that nobody reads at
// their slot (link word of a padding / ghost slot: bit i = array i is read
// there; nothing at inlet/outlet slots).  This completes the 32-byte sectors
// at the row ends, which the memory system would otherwise have to read
// back before writing them, at no extra instructions per warp.
template <int P, bool GHOST1, bool WIDE, bool WALLQ, int AX>
__device__ __forceinline__ void cell_update(const StepArgs &a, int row, int x, bool fluid, int qk, double (&hv)[6]) {
    using R = typename Storage<P>::R;
    int nb[9];
    load_row(a.row_nb, row, nb);
    const int slot = nb[4] + x;
    const uint32_t m = __ldg(a.mask + slot);  // needed after the collision only
    const uint32_t links = fluid ? (m & LINK_MASK) : 0u;
    const uint32_t own = fluid ? (LINK_MASK | OWN_FLUID)
                               : (((m >> TYPE_SHIFT) & 3u) == TYPE_PAD ? (~m & LINK_MASK) : 0u);
    R d[27];
    R rho, ux, uy, uz;
    constexpr bool RAW = GHOST1 && Storage<P>::SCALED;  // FP16 scale folded into the collision
    gather<P, WIDE, AX, RAW>(a, nb, x, d);
    if constexpr (WALLQ) interpolate_walls<P, WIDE, RAW>(a, qk, slot, links, d);
    if constexpr (GHOST1) {
        const LineStore<P, WIDE, RAW, AX> sink{a, nb, x, slot, links, own};
        collide_ghost1<R, RAW, LineStore<P, WIDE, RAW, AX>>(d, flow<R>(a).omega, rho, ux, uy, uz, R(a.inv_scale),
                                                            R(a.scale), &sink);
    } else {
        if (!fluid) return;
        collide<P, GHOST1>(d, flow<R>(a), rho, ux, uy, uz, a, slot);
        store_cell_state<P, WIDE, AX, RAW>(a, nb, x, slot, links, d);
    }
    if (fluid) record_cell(a, slot, rho, ux, uy, uz, hv);
}

template <int P, bool GHOST1, bool WIDE, int AX>
__device__ __forceinline__ void fluid_cell(const StepArgs &a, int chunk, int lane, double (&hv)[6]) {
    const int2 ch = __ldg(a.chunks + chunk);
    const uint32_t cw = (uint32_t)ch.y;
    const bool fluid = (cw >> (CHUNK_LANES_SHIFT + lane)) & 1u;
    cell_update<P, GHOST1, WIDE, false, AX>(a, ch.x, (int)(cw & CHUNK_X0_MASK) + lane, fluid, -1, hv);
}

// Fluid lane of the step kernel with a warp-uniform fast path (default ghost
// rates, 32-bit offsets, FP32 / FP16S).  With rows along the flow axis most
// warps hold 32 fluid cells none of which has a wall link (or, on a periodic
// row axis, sits at a row end); such a warp stores every cell's 27 values
// into its own slots and skips the line sink's per-value predicates,
// ghost-slot stores and wrap-around copies.  The gather is the same on both paths, so it
// is issued before the vote.  Every lane of the warp must call this (lanes
// past the last chunk take part in the vote only).
template <int P, int AX>
__device__ __forceinline__ void fluid_lane_voted(const StepArgs &a, int chunk, int lane, double (&hv)[6]) {
    using R = typename Storage<P>::R;
    constexpr bool RAW = Storage<P>::SCALED;
    const bool valid = chunk < a.nchunks;
    int nb[9];
    R d[27];
    int x = 0, slot = 0;
    uint32_t m = 0u;
    bool fluid = false;
    if (valid) {
        const int2 ch = __ldg(a.chunks + chunk);
        const uint32_t cw = (uint32_t)ch.y;
        fluid = (cw >> (CHUNK_LANES_SHIFT + lane)) & 1u;
        x = (int)(cw & CHUNK_X0_MASK) + lane;
        load_row(a.row_nb, ch.x, nb);
        slot = nb[4] + x;
        gather<P, false, AX, RAW>(a, nb, x, d);
        m = __ldg(a.mask + slot);
    }
    const bool row_end = a.periodic_row && (x == 0 || x == a.n_row - 1);  // writes wrap-around copies
    const bool simple = fluid && (m & LINK_MASK) == 0u && !row_end;
    const bool fast = __all_sync(0xffffffffu, simple);
    if (!valid) return;
    R rho, ux, uy, uz;
    if (fast) {
        const OwnStore<P, RAW> sink{a, slot};
        collide_ghost1<R, RAW, OwnStore<P, RAW>>(d, flow<R>(a).omega, rho, ux, uy, uz, R(a.inv_scale), R(a.scale),
                                                 &sink);
    } else {
        const uint32_t links = fluid ? (m & LINK_MASK) : 0u;
        const uint32_t own = fluid ? (LINK_MASK | OWN_FLUID)
                                   : (((m >> TYPE_SHIFT) & 3u) == TYPE_PAD ? (~m & LINK_MASK) : 0u);
        const LineStore<P, false, RAW, AX> sink{a, nb, x, slot, links, own};
        collide_ghost1<R, RAW, LineStore<P, false, RAW, AX>>(d, flow<R>(a).omega, rho, ux, uy, uz,
                                                             R(a.inv_scale), R(a.scale), &sink);
    }
    if (fluid) record_cell(a, slot, rho, ux, uy, uz, hv);
}

// Update of wall cell k of the interpolated-wall list (x, row, slot, record):
// the same update with Bouzidi's interpolation of its wall links.  These
// cells are taken out of the chunk lanes while wall distances are set, so
// the fluid kernel keeps its plain instruction stream.
template <int P, bool GHOST1, bool WIDE, int AX>
__device__ __forceinline__ void wall_cell(const StepArgs &a, int k, double (&hv)[6]) {
    const int4 node = __ldg(a.wnodes + k);
    cell_update<P, GHOST1, WIDE, true, AX>(a, node.y, node.x, true, node.w, hv);
}

// Update of inlet/outlet node k: non-equilibrium extrapolation (Sec. 2.2)
// from the interior partner x_f, whose update is recomputed here from the
// same input state (so boundary and fluid updates are independent):
//   f*_i(x_b) = f^eq_i(rho_b, u_b) + f*_i(x_f) - f^eq_i(rho_f, u_f),
// inlet: rho_b = rho_f, u_b prescribed; outlet: rho_b = rho_out, u_b = u_f.
template <int P, bool GHOST1, bool WIDE, int AX>
__device__ __forceinline__ void boundary_node(const StepArgs &a, int k, double (&hv)[6]) {
    using R = typename Storage<P>::R;
    const int4 node = __ldg(a.bnodes + k);
    const int pos = node.x, row = node.y, slot = node.z;
    const uint32_t m = (uint32_t)node.w;
    const uint32_t type = (m >> TYPE_SHIFT) & 3u;
    const FlowParams<R> &fp = flow<R>(a);
    // box position from (row position, row): (p, a, b) = (x, y, z) or (z, x, y)
    const int ra = row % a.na_e - 1, rb = row / a.na_e - 1;
    const int x = AX == 0 ? pos : ra, y = AX == 0 ? ra : rb, z = AX == 0 ? rb : pos;
    const int dir = (int)(m >> DIR_SHIFT);
    const int nx_ = (dir == 0) - (dir == 1), ny_ = (dir == 2) - (dir == 3), nz_ = (dir == 4) - (dir == 5);
    const int xf = wrap(x + nx_, a.nx), yf = wrap(y + ny_, a.ny), zf = wrap(z + nz_, a.nz);
    const int pf = AX == 0 ? xf : zf;  // the partner in storage coordinates
    const int row_f = AX == 0 ? (yf + 1) + a.na_e * (zf + 1) : (xf + 1) + a.na_e * (yf + 1);
    int nbf[9];
    load_row(a.row_nb, row_f, nbf);
    R d[27];
    R rf, uxf, uyf, uzf, rho, ux, uy, uz;
    gather<P, WIDE, AX>(a, nbf, pf, d);
    if (a.wall_qidx) {
        const int sf = nbf[4] + pf;
        const uint32_t lf = __ldg(a.mask + sf) & LINK_MASK;
        if (lf) interpolate_walls<P, WIDE, false>(a, __ldg(a.wall_qidx + sf), sf, lf, d);
    }
    collide<P, GHOST1>(d, fp, rf, uxf, uyf, uzf, a, slot);  // the node takes its partner's stress
    if (type == TYPE_INLET) {
        R speed = fp.u_in;
        if (a.profile == LBM_PROFILE_PARABOLIC) {
            const R rx = R(x) + R(0.5) - fp.axis_x, ry = R(y) + R(0.5) - fp.axis_y;
            const R r2 = rx * rx + ry * ry;
            speed = R(2) * fp.u_in * (R(1) - R(4) * r2 / (fp.d_in * fp.d_in));
        }
        rho = rf;
        ux = speed * R(nx_);
        uy = speed * R(ny_);
        uz = speed * R(nz_);
        if (fp.noise_amp != R(0)) {
            const int64_t node_id = (int64_t)x + (int64_t)a.nx * ((int64_t)y + (int64_t)a.ny * z);
            const R amp = fp.noise_amp * fp.u_in;
            ux += amp * inlet_noise<R>(a.seed, a.t_new, node_id, 0);
            uy += amp * inlet_noise<R>(a.seed, a.t_new, node_id, 1);
            uz += amp * inlet_noise<R>(a.seed, a.t_new, node_id, 2);
        }
        if (a.t_new < a.inlet_ramp) {  // smooth start: u_b r(t), r = s^2 (3 - 2 s), s = t / T
            const R sr = R(a.t_new) / R(a.inlet_ramp), r = sr * sr * (R(3) - R(2) * sr);
            ux *= r;
            uy *= r;
            uz *= r;
        }
    } else {
        rho = fp.rho_out;
        ux = uxf;
        uy = uyf;
        uz = uzf;
    }
    add_eq_difference<R>(rho, ux, uy, uz, rf, uxf, uyf, uzf, d);
    int nb[9];
    load_row(a.row_nb, row, nb);
    store_cell_state<P, WIDE, AX>(a, nb, pos, slot, 0u, d);
    record_cell(a, slot, rho, ux, uy, uz, hv);
}

// Largest span one population's L2 prefetch may cover (bytes).
constexpr int64_t PREFETCH_MAX_BYTES = 16384;

// L2 prefetch of the pull sources of fluid block tb, population i.  The
// block's chunks cover rows r0..r1 in storage order, and the rows that
// population i pulls from, r + (cy, cz) for every r, are stored back to back
// in the same order, so its sources (slots nb_r[j] + x - cx) lie in one span
// from the first chunk's first lane to the last chunk's last lane.  The span
// is widened to 16-byte bounds, which stay inside the buffer margins.  Spans
// that wrap around a periodic y or z face (reversed or very long) are
// skipped: a prefetch only moves data, never changes a result.
template <int P, int AX>
__device__ __forceinline__ void prefetch_block_sources(const StepArgs &a, int tb, int i) {
    using T = typename Storage<P>::T;
    const int c0 = tb * (STEP_THREADS / CHUNK);
    if (tb < 0 || c0 >= a.nchunks) return;
    const int c1 = min(c0 + STEP_THREADS / CHUNK, a.nchunks) - 1;
    const int2 h0 = __ldg(a.chunks + c0), h1 = __ldg(a.chunks + c1);
    const int j = row_line<AX>(i), cx = c_row<AX>(i);
    const int *rn = reinterpret_cast<const int *>(a.row_nb);
    const int b0 = __ldg(rn + (int64_t)ROW_RECORD_INTS * h0.x + j);
    const int b1 = __ldg(rn + (int64_t)ROW_RECORD_INTS * h1.x + j);
    const int64_t s0 = (int64_t)b0 + (int)((uint32_t)h0.y & CHUNK_X0_MASK) - cx;
    const int64_t s1 = (int64_t)b1 + (int)((uint32_t)h1.y & CHUNK_X0_MASK) + CHUNK - cx;
    if (s1 <= s0 || (s1 - s0) * (int64_t)sizeof(T) > PREFETCH_MAX_BYTES) return;
    const char *arr = static_cast<const char *>(a.fin) + (int64_t)i * a.stride * (int64_t)sizeof(T);
    const uintptr_t lo = (uintptr_t)(arr + s0 * (int64_t)sizeof(T)) & ~(uintptr_t)15;
    const uintptr_t hi = ((uintptr_t)(arr + s1 * (int64_t)sizeof(T)) + 15) & ~(uintptr_t)15;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((uint32_t)(hi - lo)) : "memory");
}

// One time step of every fluid cell of one lattice.  The last warp of each
// block also prefetches the pull sources of block blockIdx.x +
// a.prefetch_ahead into L2 (one bulk prefetch per population), so that the
// gathers of later blocks find their rows in L2 instead of waiting on HBM.
template <int P, bool GHOST1, bool WIDE, int AX>
__global__ void __launch_bounds__(STEP_THREADS, P == 0 ? 1 : LBM_STEP_MIN_BLOCKS) k_step(const StepArgs a) {
    double hv[6] = {0, 0, 0, 0, 0, 0};
    if (LBM_FUSE_BOUNDARY && P == 1 && (int)blockIdx.x >= a.fluid_blocks) {  // inlet/outlet nodes, trailing blocks
        const int k = ((int)blockIdx.x - a.fluid_blocks) * STEP_THREADS + (int)threadIdx.x;
        if (k < a.nbnodes) boundary_node<P, GHOST1, WIDE, AX>(a, k, hv);
    } else {
        const int gt = blockIdx.x * STEP_THREADS + threadIdx.x;
        const int chunk = gt / CHUNK;
        if constexpr (LBM_FAST_PATH && GHOST1 && !WIDE && P != 0)
            fluid_lane_voted<P, AX>(a, chunk, gt % CHUNK, hv);  // every lane of the block calls it
        else if (chunk < a.nchunks)
            fluid_cell<P, GHOST1, WIDE, AX>(a, chunk, gt % CHUNK, hv);
        if (a.prefetch_ahead > 0) {
            const int i = (int)threadIdx.x - (STEP_THREADS - 32);
            if (i >= 0 && i < 27) prefetch_block_sources<P, AX>(a, (int)blockIdx.x + a.prefetch_ahead, i);
        }
    }
    if (a.flags & STEP_REDUCE) block_reduce_write(hv, a.partials);
}

// One time step of the cells with interpolated walls (see wall_cell); its
// partial sums follow those of the fluid and inlet/outlet kernels.
template <int P, bool GHOST1, bool WIDE, int AX>
__global__ void __launch_bounds__(STEP_THREADS, P == 0 ? 1 : LBM_STEP_MIN_BLOCKS_WALLQ) k_wall(const StepArgs a) {
    const int k = blockIdx.x * STEP_THREADS + threadIdx.x;
    double hv[6] = {0, 0, 0, 0, 0, 0};
    if (k < a.nwnodes) wall_cell<P, GHOST1, WIDE, AX>(a, k, hv);
    if (a.flags & STEP_REDUCE) {
        const int before = a.fluid_blocks + (a.nbnodes + STEP_THREADS - 1) / STEP_THREADS;
        block_reduce_write(hv, a.partials + (size_t)before * REDUCE_SLOTS);
    }
}

// One time step of every inlet/outlet node of one lattice (when they do not
// ride in the trailing blocks of k_step).
template <int P, bool GHOST1, bool WIDE, int AX>
__global__ void __launch_bounds__(STEP_THREADS) k_boundary(const StepArgs a) {
    const int k = blockIdx.x * STEP_THREADS + threadIdx.x;
    double hv[6] = {0, 0, 0, 0, 0, 0};
    if (k < a.nbnodes) boundary_node<P, GHOST1, WIDE, AX>(a, k, hv);
    if (a.flags & STEP_REDUCE) block_reduce_write(hv, a.partials + (size_t)a.fluid_blocks * REDUCE_SLOTS);
}

// -------------------------------------------------------- tile fluid kernel
//
// Variant of the fluid kernel (default ghost rates, 32-bit offsets, FP32 /
// FP16S) over tile records instead of chunk records: one warp updates one
// tile, up to 32 consecutive cells of a row.  Its record (p0, lanes, the
// nine neighbour-row bases) is one 48-byte load with no dependent index
// load before the gather.  A "fast" tile (32 fluid cells, no wall link, no
// wrap-around copy; flagged when the index is built) stores through shared
// memory: each lane writes its 27 values at fixed offsets, and the warp
// writes every population's 32 consecutive own slots as 16-byte stores, so
// the 27 per-value address computations of the line sink disappear.  Other
// tiles load their link words and use the line sink.

template <int P>
struct TileOut {
    using T = typename Storage<P>::T;
    static constexpr int S = (int)sizeof(T);
    static constexpr int PIECE = 16 / S;          // elements of one 16-byte store
    static constexpr int PIECES = 32 / PIECE;     // 16-byte pieces of one population's 32 outputs
    static constexpr int ELEMS = 27 * 32;         // a warp's staged outputs
};

// Output sink of a fast tile: value i of lane l goes to out[i * 32 + l] in
// the warp's shared-memory slice (out points at lane l's first element).
template <int P, bool RAW>
struct SharedStore {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    const StepArgs &a;
    int slot;
    T *out;
    __device__ __forceinline__ void put(int i, R v) const {
        if constexpr (RAW)
            S::store_raw(out + 32 * i, v);
        else
            S::store(out + 32 * i, v, R(a.scale));
    }
    __device__ __forceinline__ void moments(R omega, const R (&a2)[6]) const { record_stress(a, slot, omega, a2); }
    __device__ __forceinline__ void operator()(int j, R vm, R v0, R vp) const {
        put(3 * j, vm);
        put(3 * j + 1, v0);
        put(3 * j + 2, vp);
    }
};

// One warp's update of tile t (lane = the warp lane, out = the warp's
// shared-memory slice of TileOut<P>::ELEMS elements).
template <int P, int AX>
__device__ __forceinline__ void tile_update(const StepArgs &a, int t, int lane, typename TileOut<P>::T *out,
                                            double (&hv)[6]) {
    using O = TileOut<P>;
    using T = typename O::T;
    using R = typename Storage<P>::R;
    constexpr bool RAW = Storage<P>::SCALED;
    const int4 *rec = reinterpret_cast<const int4 *>(a.tiles) + 3 * (size_t)t;
    const int4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r2 = __ldg(rec + 2);
    const int nb[9] = {r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, r2.w};
    const bool fast = ((uint32_t)r0.x & TILE_FAST) != 0u;
    const int p0 = (int)((uint32_t)r0.x & CHUNK_X0_MASK);
    const int x = p0 + lane, slot = nb[4] + x;
    const bool fluid = ((uint32_t)r0.y >> lane) & 1u;
    R d[27];
    gather<P, false, AX, RAW>(a, nb, x, d);  // every lane's pulls lie inside the buffer margins
    R rho, ux, uy, uz;
    if (fast) {
        const SharedStore<P, RAW> sink{a, slot, out + lane};
        collide_ghost1<R, RAW, SharedStore<P, RAW>>(d, flow<R>(a).omega, rho, ux, uy, uz, R(a.inv_scale),
                                                    R(a.scale), &sink);
        __syncwarp();
        // piece q = 4 i + k (FP16S) / 8 i + k (FP32): elements 16k/S.. of population i,
        // at shared offset 16 q bytes and at own slots nb[4] + p0 + k PIECE
        T *fout = static_cast<T *>(a.fout) + (nb[4] + p0);
#pragma unroll
        for (int q0 = 0; q0 < 27 * O::PIECES; q0 += 32) {
            const int q = q0 + lane;
            if (q < 27 * O::PIECES) {
                const int4 v = reinterpret_cast<const int4 *>(out)[q];
                const int i = q / O::PIECES, k = q % O::PIECES;
                *reinterpret_cast<int4 *>(fout + elem<false>(i, a.stride, k * O::PIECE)) = v;
            }
        }
        __syncwarp();
    } else {
        const bool present = ((uint32_t)r0.z >> lane) & 1u;
        const uint32_t m = present ? __ldg(a.mask + slot) : 0u;
        const uint32_t links = fluid ? (m & LINK_MASK) : 0u;
        const uint32_t own = fluid ? (LINK_MASK | OWN_FLUID)
                                   : (present && ((m >> TYPE_SHIFT) & 3u) == TYPE_PAD ? (~m & LINK_MASK) : 0u);
        const LineStore<P, false, RAW, AX> sink{a, nb, x, slot, links, own};
        collide_ghost1<R, RAW, LineStore<P, false, RAW, AX>>(d, flow<R>(a).omega, rho, ux, uy, uz, R(a.inv_scale),
                                                             R(a.scale), &sink);
    }
    if (fluid) record_cell(a, slot, rho, ux, uy, uz, hv);
}

template <int P, int AX>
__global__ void __launch_bounds__(STEP_THREADS, LBM_STEP_MIN_BLOCKS) k_step_tiles(const StepArgs a) {
    using O = TileOut<P>;
    __shared__ __align__(16) typename O::T staged_out[STEP_THREADS / 32][O::ELEMS];
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const int t = (int)blockIdx.x * (STEP_THREADS / 32) + warp;
    double hv[6] = {0, 0, 0, 0, 0, 0};
    if (t < a.ntiles) tile_update<P, AX>(a, t, lane, staged_out[warp], hv);  // uniform over the warp
    if (a.flags & STEP_REDUCE) block_reduce_write(hv, a.partials);
}

// ------------------------------------------------ pair fluid kernel (FP16S)
//
// Fast tiles of an FP16S lattice (32 fluid cells, no wall link, no
// wrap-around copy) with two adjacent cells per thread: 16 threads per
// tile, thread k updates cells x = p0 + 2k and x + 1.  The collision runs on
// the packed FP32 pipe across the pair (one instruction for both cells); its
// 27 inputs stay FP16 pairs until the moment pass converts them; the pull
// of each line along the row (c = 0 along the row axis) is one aligned
// 32-bit load of both cells' values, the other two are two 16-bit loads;
// each output is one 32-bit store of both cells' own slots.  Every thread
// holds two cells, so the kernel runs at fewer resident warps than the
// one-cell kernels with the same bytes in flight per SM.
#ifndef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_MIN_BLOCKS 5
#endif

struct Half2ToF2 {
    __device__ __forceinline__ F2 operator()(__half2 h) const { return F2(__half22float2(h)); }
};

// Pull gather of the pair (x, x + 1), x even: d[i] = FP16 pulls of both cells.
template <int AX>
__device__ __forceinline__ void gather_pair(const StepArgs &a, const int (&nb)[9], int x, __half2 (&d)[27]) {
    const __half *fin = static_cast<const __half *>(a.fin);
    const uint32_t st = (uint32_t)a.stride;
    constexpr int dk = line_pop<AX>(0, 1) - line_pop<AX>(0, 0);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const __half *pj = fin + ((uint32_t)line_pop<AX>(j, 0) * st + (uint32_t)(nb[j] + x));
        // c_row = -1: pulls from x + 1, x + 2
        d[line_pop<AX>(j, 0)] = __halves2half2(__ldg(pj + 1), __ldg(pj + 2));
        // c_row = 0: pulls from x, x + 1, one aligned 32-bit load
        d[line_pop<AX>(j, 1)] = __ldg(reinterpret_cast<const __half2 *>(pj + dk * st));
        // c_row = +1: pulls from x - 1, x
        d[line_pop<AX>(j, 2)] = __halves2half2(__ldg(pj + 2 * dk * st - 1), __ldg(pj + 2 * dk * st));
    }
}

// Viscous stress of the pair's two cells (statistics sample steps).
__device__ __forceinline__ void record_stress_pair(const StepArgs &a, int slot, F2 omega, const F2 (&a2)[6]) {
    if ((a.flags & (STEP_STATS | STEP_STATS_FULL)) != (STEP_STATS | STEP_STATS_FULL)) return;
    float ax[6], ay[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) ax[q] = a2[q].v.x, ay[q] = a2[q].v.y;
    record_stress(a, slot, omega.v.x, ax);
    record_stress(a, slot + 1, omega.v.y, ay);
}

// Output sink of a fast tile: both cells' values of population i as one FP16
// pair at their own slots (slot even), already scaled by the collision.
struct PairStore {
    const StepArgs &a;
    int slot;
    __device__ __forceinline__ void moments(F2 omega, const F2 (&a2)[6]) const {
        record_stress_pair(a, slot, omega, a2);
    }
    __device__ __forceinline__ void operator()(int j, F2 vm, F2 v0, F2 vp) const {
        const uint32_t st = (uint32_t)a.stride;
        __half *pj = static_cast<__half *>(a.fout) + ((uint32_t)(3 * j) * st + (uint32_t)slot);
        *reinterpret_cast<__half2 *>(pj) = __float22half2_rn(vm.v);
        *reinterpret_cast<__half2 *>(pj + st) = __float22half2_rn(v0.v);
        *reinterpret_cast<__half2 *>(pj + 2 * st) = __float22half2_rn(vp.v);
    }
};

// Half a warp's update of fast tile t with two cells per thread (k: the
// pair within the tile).
template <int AX>
__device__ __forceinline__ void pair_update(const StepArgs &a, int t, int k, double (&hv)[6]) {
    const int4 *rec = reinterpret_cast<const int4 *>(a.tiles) + 3 * (size_t)t;
    const int4 r0 = __ldg(rec), r1 = __ldg(rec + 1), r2 = __ldg(rec + 2);
    const int nb[9] = {r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, r2.w};
    const int x = (int)((uint32_t)r0.x & CHUNK_X0_MASK) + 2 * k, slot = nb[4] + x;
    __half2 d[27];
    gather_pair<AX>(a, nb, x, d);
    F2 m[10], rho, ux, uy, uz;
    ghost1_sums(d, Half2ToF2{}, m);
    ghost1_finish<F2, true>(m, F2(a.pf.omega), rho, ux, uy, uz, F2(a.inv_scale), F2(a.scale), PairStore{a, slot});
    double h0[6] = {0, 0, 0, 0, 0, 0}, h1[6] = {0, 0, 0, 0, 0, 0};
    record_cell(a, slot, rho.v.x, ux.v.x, uy.v.x, uz.v.x, h0);
    record_cell(a, slot + 1, rho.v.y, ux.v.y, uy.v.y, uz.v.y, h1);
#pragma unroll
    for (int q = 0; q < 6; ++q) hv[q] = q == 4 ? fmax(h0[q], h1[q]) : h0[q] + h1[q];
}

// FP16S pair kernel: one pair of fast tiles per warp (in row order), 16
// threads per tile, two cells per thread.  Every other cell of the lattice
// is updated by the chunk kernel over the remaining chunks, in a launch of
// its own: one instruction stream per kernel, each at its own register
// budget.
template <int AX>
__global__ void __launch_bounds__(STEP_THREADS, LBM_PAIR_MIN_BLOCKS) k_step_pairs(const StepArgs a) {
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    const int w = (int)blockIdx.x * (STEP_THREADS / 32) + warp;
    double hv[6] = {0, 0, 0, 0, 0, 0};
    if (w < a.nitems) {
        const int2 item = __ldg(a.items + w);
        pair_update<AX>(a, lane < 16 ? item.x : item.y, lane & 15, hv);
    }
    if (a.flags & STEP_REDUCE) block_reduce_write(hv, a.partials);
}

// ---------------------------------------------------------- utility kernels

template <int P>
__device__ __forceinline__ void load_cell(const void *f, int64_t stride, int slot, float inv_scale,
                                          double (&d)[27]) {
    using S = Storage<P>;
    const typename S::T *p = static_cast<const typename S::T *>(f);
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        if constexpr (P == 2)
            d[i] = (double)__half2float(p[(int64_t)i * stride + slot]) * (double)inv_scale;
        else
            d[i] = (double)p[(int64_t)i * stride + slot];
    }
}

__device__ __forceinline__ void moments_of(const double (&d)[27], double &rho, double &ux, double &uy,
                                           double &uz) {
    double drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        drho += d[i];
        jx += cx_of(i) * d[i];
        jy += cy_of(i) * d[i];
        jz += cz_of(i) * d[i];
    }
    rho = 1.0 + drho;
    ux = jx / rho;
    uy = jy / rho;
    uz = jz / rho;
}

// Health reduction of a stored state (mass, momentum, max |u|, non-finite count).
template <int P>
__global__ void __launch_bounds__(STEP_THREADS) k_reduce(const void *f, const int32_t *slot_of_active, int64_t n,
                                                         int64_t stride, float inv_scale, double *partials) {
    const int64_t k = (int64_t)blockIdx.x * STEP_THREADS + threadIdx.x;
    double hv[6] = {0, 0, 0, 0, 0, 0};
    if (k < n) {
        double d[27], rho, ux, uy, uz;
        load_cell<P>(f, stride, slot_of_active[k], inv_scale, d);
        moments_of(d, rho, ux, uy, uz);
        health_values(rho, ux, uy, uz, hv);
    }
    block_reduce_write(hv, partials);
}

// Ghost slots and periodic copies along the rows of one buffer from its
// active cells: the same writes the step kernel does after its collision,
// for a state set from the host.
template <int P, int AX>
__global__ void __launch_bounds__(STEP_THREADS) k_fill_ghosts(void *f, const uint32_t *mask, const int2 *chunks,
                                                              const int4 *row_nb, int32_t nchunks, int64_t stride,
                                                              int32_t n_row, int32_t periodic_row) {
    using T = typename Storage<P>::T;
    const int gt = blockIdx.x * STEP_THREADS + threadIdx.x;
    const int chunk = gt / CHUNK;
    if (chunk >= nchunks) return;
    const int2 ch = chunks[chunk];
    const uint32_t cw = (uint32_t)ch.y;
    const int lane = gt % CHUNK;
    if (!((cw >> (CHUNK_LANES_SHIFT + lane)) & 1u)) return;
    const int x = (int)(cw & CHUNK_X0_MASK) + lane;
    int nb[9];
    load_row(row_nb, ch.x, nb);
    const int slot = nb[4] + x;
    T *p = static_cast<T *>(f);
    const uint32_t links = mask[slot] & LINK_MASK;
#pragma unroll
    for (int i = 0; i < 27; ++i)
        if (links & (1u << i))
            p[(int64_t)i * stride + nb[row_line<AX>(i)] + x - c_row<AX>(i)] = p[(int64_t)(26 - i) * stride + slot];
    if (periodic_row) {
        if (x == n_row - 1)
#pragma unroll
            for (int i = 0; i < 27; ++i)
                if (c_row<AX>(i) == 1) p[(int64_t)i * stride + nb[4] - 1] = p[(int64_t)i * stride + slot];
        if (x == 0)
#pragma unroll
            for (int i = 0; i < 27; ++i)
                if (c_row<AX>(i) == -1) p[(int64_t)i * stride + nb[4] + n_row] = p[(int64_t)i * stride + slot];
    }
}

// Periodic copies along the rows of the inlet/outlet nodes.
template <int P, int AX>
__global__ void __launch_bounds__(STEP_THREADS) k_fill_periodic_nodes(void *f, const int4 *bnodes, int32_t nbnodes,
                                                                      const int4 *row_nb, int64_t stride,
                                                                      int32_t n_row) {
    using T = typename Storage<P>::T;
    const int k = blockIdx.x * STEP_THREADS + threadIdx.x;
    if (k >= nbnodes) return;
    const int4 node = bnodes[k];
    const int x = node.x, slot = node.z;
    const int base = row_nb[3 * node.y + 1].x;
    T *p = static_cast<T *>(f);
    if (x == n_row - 1)
#pragma unroll
        for (int i = 0; i < 27; ++i)
            if (c_row<AX>(i) == 1) p[(int64_t)i * stride + base - 1] = p[(int64_t)i * stride + slot];
    if (x == 0)
#pragma unroll
        for (int i = 0; i < 27; ++i)
            if (c_row<AX>(i) == -1) p[(int64_t)i * stride + base + n_row] = p[(int64_t)i * stride + slot];
}

template <int P>
__global__ void k_moments(const void *f, const int32_t *slot_of_active, int64_t n, int64_t stride, float inv_scale,
                          double *out4) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double d[27], rho, ux, uy, uz;
    load_cell<P>(f, stride, slot_of_active[k], inv_scale, d);
    moments_of(d, rho, ux, uy, uz);
    out4[4 * k] = rho;
    out4[4 * k + 1] = ux;
    out4[4 * k + 2] = uy;
    out4[4 * k + 3] = uz;
}

__device__ __forceinline__ double wd(int i) {
    return w1<double>(cx_of(i)) * w1<double>(cy_of(i)) * w1<double>(cz_of(i));
}

template <int P>
__global__ void k_get_populations(const void *f, const int32_t *slot_of_active, int64_t n, int64_t stride,
                                  float inv_scale, double *out27) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double d[27];
    load_cell<P>(f, stride, slot_of_active[k], inv_scale, d);
#pragma unroll
    for (int i = 0; i < 27; ++i) out27[27 * k + i] = wd(i) + d[i];
}

template <int P>
__device__ __forceinline__ void store_cell(void *f, int64_t stride, int slot, float scale, const double (&d)[27]) {
    using S = Storage<P>;
    typename S::T *p = static_cast<typename S::T *>(f);
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        if constexpr (P == 2)
            p[(int64_t)i * stride + slot] = __float2half_rn((float)(d[i] * (double)scale));
        else
            p[(int64_t)i * stride + slot] = (typename S::T)d[i];
    }
}

template <int P>
__global__ void k_set_populations(void *f, const int32_t *slot_of_active, int64_t n, int64_t stride, float scale,
                                  const double *in27) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double d[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) d[i] = in27[27 * k + i] - wd(i);
    store_cell<P>(f, stride, slot_of_active[k], scale, d);
}

template <int P>
__global__ void k_init_eq(void *f, const int32_t *slot_of_active, int64_t n, int64_t stride, float scale,
                          const double *rho, const double *u, double rho0, double ux0, double uy0, double uz0) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double r = rho ? rho[k] : rho0;
    const double ux = u ? u[3 * k] : ux0, uy = u ? u[3 * k + 1] : uy0, uz = u ? u[3 * k + 2] : uz0;
    double d[27];
    eq_deviation<double>(r, Axis<double>(ux), Axis<double>(uy), Axis<double>(uz), d);
    store_cell<P>(f, stride, slot_of_active[k], scale, d);
}

// --------------------------------------------------------------- launchers

inline int step_blocks(int32_t nchunks) {
    const int64_t threads = (int64_t)nchunks * CHUNK;
    return (int)((threads + STEP_THREADS - 1) / STEP_THREADS);
}

// Partial-sum slots written by the fluid kernel of one step.
template <int P>
int step_fluid_blocks(int32_t nchunks) {
    return step_blocks(nchunks);
}

template <int P>
int step_prefetch_ahead(bool ghost1, bool wide, int device) {
    int per_sm = 0, sms = 0;
    cudaError_t e;
    if (ghost1)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, wide ? k_step<P, true, true, 0> : k_step<P, true, false, 0>, STEP_THREADS, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, wide ? k_step<P, false, true, 0> : k_step<P, false, false, 0>, STEP_THREADS, 0);
    if (e != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int pct = P == 2 ? LBM_PREFETCH_AHEAD_PCT_FP16S : LBM_PREFETCH_AHEAD_PCT;
    return (int)((int64_t)per_sm * sms * pct / 100);
}

// The wall-cell and inlet/outlet kernels of a step (those not fused into
// the fluid kernel), on stream sn.
template <int P, bool G, bool WD, int AX>
void launch_node_kernels(const StepArgs &a, cudaStream_t sn, bool boundary, int &launches) {
    if (a.nwnodes > 0) {  // cells with interpolated walls
        k_wall<P, G, WD, AX><<<(a.nwnodes + STEP_THREADS - 1) / STEP_THREADS, STEP_THREADS, 0, sn>>>(a);
        ++launches;
    }
    if (boundary && a.nbnodes > 0) {
        k_boundary<P, G, WD, AX><<<(a.nbnodes + STEP_THREADS - 1) / STEP_THREADS, STEP_THREADS, 0, sn>>>(a);
        ++launches;
    }
}

// One step: the node kernels go first, on the side stream when there is one
// (forked from s and joined back into it at the end), so that their few
// long-latency blocks run beside the fluid kernel instead of after it.  All
// kernels of a step read the input buffer only and write disjoint output
// elements and partial sums, so their order does not change any result.
template <int P, bool G, bool WD, int AX>
cudaError_t launch_step_ax(const StepArgs &a, cudaStream_t s, const SideStream *side, int &launches) {
    const int bb = (int)((a.nbnodes + STEP_THREADS - 1) / STEP_THREADS);
    const bool tiled = G && !WD && P != 0 && a.tiles != nullptr;
    const bool fused = !tiled && LBM_FUSE_BOUNDARY && P == 1 && a.nchunks > 0;  // nodes in trailing blocks of k_step
    const bool nodes = a.nwnodes > 0 || (bb > 0 && !fused);
    const bool aside = nodes && side && side->stream;
    cudaStream_t sn = s;
    if (aside) {
        cudaError_t e = cudaEventRecord(side->fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side->stream, side->fork, 0);
        if (e != cudaSuccess) return e;
        sn = side->stream;
    }
    launch_node_kernels<P, G, WD, AX>(a, sn, !fused, launches);
    if constexpr (G && !WD && P != 0) {
        if (tiled) {
            if constexpr (P == 2) {
                if (a.items) {  // FP16S split: pairs of fast tiles, two cells per thread; the other chunks
                    if (a.nchunks > 0) {
                        k_step<P, G, WD, AX><<<step_blocks(a.nchunks), STEP_THREADS, 0, s>>>(a);
                        ++launches;
                    }
                    if (a.nitems > 0) {
                        StepArgs b = a;  // partial sums after the chunk kernel's
                        b.partials = a.partials + (size_t)step_blocks(a.nchunks) * REDUCE_SLOTS;
                        k_step_pairs<AX><<<tile_blocks(a.nitems), STEP_THREADS, 0, s>>>(b);
                        ++launches;
                    }
                } else if (a.ntiles > 0) {
                    k_step_tiles<P, AX><<<tile_blocks(a.ntiles), STEP_THREADS, 0, s>>>(a);
                    ++launches;
                }
            } else if (a.ntiles > 0) {
                k_step_tiles<P, AX><<<tile_blocks(a.ntiles), STEP_THREADS, 0, s>>>(a);
                ++launches;
            }
        }
    }
    if (!tiled && a.nchunks > 0) {
        k_step<P, G, WD, AX><<<step_blocks(a.nchunks) + (fused ? bb : 0), STEP_THREADS, 0, s>>>(a);
        ++launches;
    }
    if (aside) {
        cudaError_t e = cudaEventRecord(side->join, sn);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, side->join, 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int P, bool G, bool WD>
cudaError_t launch_step_rows(const StepArgs &a, cudaStream_t s, const SideStream *side, int &launches) {
    return a.row_axis == 2 ? launch_step_ax<P, G, WD, 2>(a, s, side, launches)
                           : launch_step_ax<P, G, WD, 0>(a, s, side, launches);
}

// One time step of a lattice; launches (if not NULL) is increased by the
// number of kernels launched; side (if not NULL) is the stream of the
// wall-cell and inlet/outlet kernels.
template <int P>
cudaError_t launch_step(const StepArgs &a, bool ghost1, cudaStream_t s, int *launches, const SideStream *side) {
    const bool wide = a.wide_offsets || a.stride > MAX_SLOTS_32;
    int n = 0;
    cudaError_t e;
    if (ghost1)
        e = wide ? launch_step_rows<P, true, true>(a, s, side, n) : launch_step_rows<P, true, false>(a, s, side, n);
    else
        e = wide ? launch_step_rows<P, false, true>(a, s, side, n) : launch_step_rows<P, false, false>(a, s, side, n);
    if (launches) *launches += n;
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int P>
cudaError_t launch_reduce(const void *f, const int32_t *slot_of_active, int64_t n, int64_t stride, float inv_scale,
                          double *partials, cudaStream_t s) {
    const int blocks = (int)((n + STEP_THREADS - 1) / STEP_THREADS);
    if (blocks == 0) return cudaSuccess;
    k_reduce<P><<<blocks, STEP_THREADS, 0, s>>>(f, slot_of_active, n, stride, inv_scale, partials);
    return cudaGetLastError();
}

template <int P, int AX>
void launch_fill_ghosts_ax(void *f, const uint32_t *mask, const int2 *chunks, const int4 *row_nb, int32_t nchunks,
                           const int4 *bnodes, int32_t nbnodes, int64_t stride, int32_t n_row, int32_t periodic_row,
                           cudaStream_t s) {
    const int blocks = step_blocks(nchunks);
    if (blocks > 0)
        k_fill_ghosts<P, AX><<<blocks, STEP_THREADS, 0, s>>>(f, mask, chunks, row_nb, nchunks, stride, n_row,
                                                             periodic_row);
    if (periodic_row && nbnodes > 0)
        k_fill_periodic_nodes<P, AX><<<(nbnodes + STEP_THREADS - 1) / STEP_THREADS, STEP_THREADS, 0, s>>>(
            f, bnodes, nbnodes, row_nb, stride, n_row);
}

template <int P>
cudaError_t launch_fill_ghosts(void *f, const uint32_t *mask, const int2 *chunks, const int4 *row_nb,
                               int32_t nchunks, const int4 *bnodes, int32_t nbnodes, int64_t stride, int32_t n_row,
                               int32_t periodic_row, int32_t row_axis, cudaStream_t s) {
    if (row_axis == 2)
        launch_fill_ghosts_ax<P, 2>(f, mask, chunks, row_nb, nchunks, bnodes, nbnodes, stride, n_row, periodic_row, s);
    else
        launch_fill_ghosts_ax<P, 0>(f, mask, chunks, row_nb, nchunks, bnodes, nbnodes, stride, n_row, periodic_row, s);
    return cudaGetLastError();
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <int P>
cudaError_t launch_moments(const void *f, const int32_t *soa, int64_t n, int64_t stride, float inv_scale,
                           double *out4, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_moments<P><<<grid_for(n, 256), 256, 0, s>>>(f, soa, n, stride, inv_scale, out4);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_get_populations(const void *f, const int32_t *soa, int64_t n, int64_t stride, float inv_scale,
                                   double *out27, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_get_populations<P><<<grid_for(n, 128), 128, 0, s>>>(f, soa, n, stride, inv_scale, out27);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_set_populations(void *f, const int32_t *soa, int64_t n, int64_t stride, float scale,
                                   const double *in27, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_set_populations<P><<<grid_for(n, 128), 128, 0, s>>>(f, soa, n, stride, scale, in27);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_init_eq(void *f, const int32_t *soa, int64_t n, int64_t stride, float scale, const double *rho,
                           const double *u, double rho0, double ux, double uy, double uz, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_init_eq<P><<<grid_for(n, 128), 128, 0, s>>>(f, soa, n, stride, scale, rho, u, rho0, ux, uy, uz);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE(P)                                                                                         \
    template cudaError_t launch_step<P>(const StepArgs &, bool, cudaStream_t, int *, const SideStream *);                                     \
    template int step_fluid_blocks<P>(int32_t);                                                                     \
    template int step_prefetch_ahead<P>(bool, bool, int);                                                          \
    template cudaError_t launch_reduce<P>(const void *, const int32_t *, int64_t, int64_t, float, double *,       \
                                          cudaStream_t);                                                           \
    template cudaError_t launch_fill_ghosts<P>(void *, const uint32_t *, const int2 *, const int4 *, int32_t,      \
                                               const int4 *, int32_t, int64_t, int32_t, int32_t, int32_t,          \
                                               cudaStream_t);                                                      \
    template cudaError_t launch_moments<P>(const void *, const int32_t *, int64_t, int64_t, float, double *,       \
                                           cudaStream_t);                                                          \
    template cudaError_t launch_get_populations<P>(const void *, const int32_t *, int64_t, int64_t, float,         \
                                                   double *, cudaStream_t);                                        \
    template cudaError_t launch_set_populations<P>(void *, const int32_t *, int64_t, int64_t, float,               \
                                                   const double *, cudaStream_t);                                  \
    template cudaError_t launch_init_eq<P>(void *, const int32_t *, int64_t, int64_t, float, const double *,       \
                                           const double *, double, double, double, double, cudaStream_t);

}  // namespace lbm
