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
// GB300 design: one thread per active cell, pull scheme over a fluid-only
// slot layout (rows of x-contiguous cells), structure-of-arrays populations
// stored as deviations from the lattice weights.  Because T(u) is the tensor
// product of three 1-D 3x3 transforms, T and its inverse are applied as a
// cascade of 1-D passes in registers; with the default ghost rates only the
// six second-order central moments survive relaxation and the inverse is the
// product-form equilibrium plus six correction terms.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "lbm_internal.h"

namespace lbm {

// ------------------------------------------------------------- storage types

template <int P>
struct Storage;

template <>
struct Storage<0> {  // FP64 deviations
    using T = double;
    using R = double;
    static __device__ __forceinline__ R load(const T *p, R) { return __ldg(p); }
    static __device__ __forceinline__ void store(T *p, R v, R) { *p = v; }
};

template <>
struct Storage<1> {  // FP32 deviations
    using T = float;
    using R = float;
    static __device__ __forceinline__ R load(const T *p, R) { return __ldg(p); }
    static __device__ __forceinline__ void store(T *p, R v, R) { *p = v; }
};

template <>
struct Storage<2> {  // FP16 (f - w) * s, FP32 arithmetic
    using T = __half;
    using R = float;
    static __device__ __forceinline__ R load(const T *p, R inv_s) { return __half2float(__ldg(p)) * inv_s; }
    static __device__ __forceinline__ void store(T *p, R v, R s) { *p = __float2half_rn(v * s); }
};

// ----------------------------------------------------------------- stencil

__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz_of(int i) { return i / 9 - 1; }

// 1-D Gauss-Hermite weights of the third-order quadrature (Appendix A).
template <class R>
__device__ __forceinline__ R w1(int c) { return c == 0 ? R(2) / R(3) : R(1) / R(6); }

template <class R>
__device__ __forceinline__ R theta0() { return R(1) / R(3); }

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

// --------------------------------------------------------------- collision

// Collision with the default ghost rates (all 1).  d holds f_i - w_i on entry
// and f*_i - w_i on exit; rho, u receive the (conserved) moments.
template <class R>
__device__ __forceinline__ void collide_ghost1(R (&d)[27], R omega, R &rho, R &ux, R &uy, R &uz) {
    // x-pass of the moment cascade: per (cy, cz) line, sums weighted by 1, cx, cx^2.
    R s0[9], s1[9], s2[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const R a = d[3 * j], b = d[3 * j + 1], c = d[3 * j + 2];
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
    rho = R(1) + drho;
    const R inv = R(1) / rho;
    ux = jx * inv;
    uy = jy * inv;
    uz = jz * inv;
    // Second-order central Hermite moments sum_i ((c-u)_a (c-u)_b - theta0 delta_ab) f_i,
    // from the deviation moments (sum c_a c_b w = theta0 delta_ab).
    const R th = theta0<R>();
    const R k = R(1) - omega;
    const R Axx = k * (pxx - rho * ux * ux - th * drho);
    const R Ayy = k * (pyy - rho * uy * uy - th * drho);
    const R Azz = k * (pzz - rho * uz * uz - th * drho);
    const R Axy = k * (pxy - rho * ux * uy);
    const R Axz = k * (pxz - rho * ux * uz);
    const R Ayz = k * (pyz - rho * uy * uz);
    // Inverse: f* = rho prod g0 + sum over the six relaxed second-order moments
    // of A_m prod_a g_{m_a}; orders 1 and 3..6 are zero after relaxation.
    const Axis<R> X(ux), Y(uy), Z(uz);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int cy = j % 3 - 1, cz = j / 3 - 1;
        const R wy = w1<R>(cy), wz = w1<R>(cz);
        const R gy0 = Y.g0[cy + 1], gz0 = Z.g0[cz + 1], gy1 = Y.g1[cy + 1], gz1 = Z.g1[cz + 1];
        const R E = gy0 * gz0;
        const R D = Y.d[cy + 1] * gz0 + wy * Z.d[cz + 1];
        const R C0 = Ayy * g2<R>(cy) * gz0 + Azz * gy0 * g2<R>(cz) + Ayz * gy1 * gz1;
        const R C1 = Axy * gy1 * gz0 + Axz * gy0 * gz1;
        const R C2 = Axx * E;
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx) {
            const R wx = w1<R>(cx);
            d[3 * j + cx + 1] = drho * (wx * wy * wz) + rho * (X.d[cx + 1] * E + wx * D) +
                                X.g0[cx + 1] * C0 + X.g1[cx + 1] * C1 + g2<R>(cx) * C2;
        }
    }
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
template <class R>
__device__ __forceinline__ void collide_general(R (&d)[27], R omega, const R (&ghost)[4], R &rho, R &ux,
                                                R &uy, R &uz) {
    R drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        drho += d[i];
        if (cx_of(i)) jx += cx_of(i) > 0 ? d[i] : -d[i];
        if (cy_of(i)) jy += cy_of(i) > 0 ? d[i] : -d[i];
        if (cz_of(i)) jz += cz_of(i) > 0 ? d[i] : -d[i];
    }
    rho = R(1) + drho;
    const R inv = R(1) / rho;
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

// Pull gather of cell (x, y, z) at storage slot `slot` with link word m:
// d_i = f*_i(x - c_i), or the halfway bounce-back f*_{26-i}(x) (Bouzidi's
// interpolated bounce-back at q = 1/2, Sec. 2.2) when bit i of m is set.
template <int P>
__device__ __forceinline__ void gather(const StepArgs &a, int x, int y, int z, int slot, uint32_t m,
                                       typename Storage<P>::R (&d)[27]) {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    const T *fin = static_cast<const T *>(a.fin);
    const R inv_s = R(a.inv_scale);
    int rb[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int ys = wrap(y - (j % 3 - 1), a.ny), zs = wrap(z - (j / 3 - 1), a.nz);
        rb[j] = __ldg(a.row_base + zs * a.ny + ys);
    }
    const int xs[3] = {wrap(x + 1, a.nx), x, wrap(x - 1, a.nx)};
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const int j = i / 3;
        const bool bb = (m >> i) & 1u;
        const int64_t off = bb ? (int64_t)(26 - i) * a.stride + slot
                               : (int64_t)i * a.stride + (rb[j] + xs[i % 3]);
        d[i] = S::load(fin + off, inv_s);
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
    __shared__ double sh[STEP_THREADS / 32][6];
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

// One time step over all active cells (Sec. 2.1 evolution equation, pull
// form).  Fluid cells gather + collide.  Inlet/outlet cells apply the
// non-equilibrium extrapolation of Sec. 2.2 with their interior partner x_f,
// whose update they recompute in place (same step, no second kernel):
//   f*_i(x_b) = f^eq_i(rho_b, u_b) + f*_i(x_f) - f^eq_i(rho_f, u_f),
// inlet: rho_b = rho_f, u_b prescribed; outlet: rho_b = rho_out, u_b = u_f.
template <int P, bool GHOST1>
__global__ void __launch_bounds__(STEP_THREADS) k_step(const StepArgs a) {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    const int gt = blockIdx.x * STEP_THREADS + threadIdx.x;
    const int chunk = gt / CHUNK;
    double hv[6] = {0, 0, 0, 0, 0, 0};
    if (chunk < a.nchunks) {
        const int2 ch = __ldg(a.chunks + chunk);
        const int row = ch.x;
        const int x = ch.y + (gt % CHUNK);
        const int y = row % a.ny, z = row / a.ny;
        const int slot = __ldg(a.row_base + row) + x;
        const uint32_t m = __ldg(a.mask + slot);
        const uint32_t type = (m >> TYPE_SHIFT) & 3u;
        if (type != TYPE_PAD) {
            R d[27];
            R rho, ux, uy, uz;
            const R omega = R(a.omega);
            R ghost[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) ghost[q] = R(a.ghost[q]);
            if (type == TYPE_FLUID) {
                gather<P>(a, x, y, z, slot, m, d);
                if (GHOST1)
                    collide_ghost1<R>(d, omega, rho, ux, uy, uz);
                else
                    collide_general<R>(d, omega, ghost, rho, ux, uy, uz);
            } else {
                const int dir = (int)(m >> DIR_SHIFT);
                const int nx_ = (dir == 0) - (dir == 1), ny_ = (dir == 2) - (dir == 3), nz_ = (dir == 4) - (dir == 5);
                const int xf = wrap(x + nx_, a.nx), yf = wrap(y + ny_, a.ny), zf = wrap(z + nz_, a.nz);
                const int slot_f = __ldg(a.row_base + zf * a.ny + yf) + xf;
                const uint32_t mf = __ldg(a.mask + slot_f);
                R rf, uxf, uyf, uzf;
                gather<P>(a, xf, yf, zf, slot_f, mf, d);
                if (GHOST1)
                    collide_ghost1<R>(d, omega, rf, uxf, uyf, uzf);
                else
                    collide_general<R>(d, omega, ghost, rf, uxf, uyf, uzf);
                if (type == TYPE_INLET) {
                    R speed = R(a.u_in);
                    if (a.profile == LBM_PROFILE_PARABOLIC) {
                        const R rx = R(x) + R(0.5) - R(a.axis_x), ry = R(y) + R(0.5) - R(a.axis_y);
                        const R r2 = rx * rx + ry * ry;
                        const R din = R(a.d_in);
                        speed = R(2) * R(a.u_in) * (R(1) - R(4) * r2 / (din * din));
                    }
                    rho = rf;
                    ux = speed * R(nx_);
                    uy = speed * R(ny_);
                    uz = speed * R(nz_);
                    if (a.noise_amp != 0.0) {
                        const int64_t node = (int64_t)x + (int64_t)a.nx * ((int64_t)y + (int64_t)a.ny * z);
                        const R amp = R(a.noise_amp) * R(a.u_in);
                        ux += amp * inlet_noise<R>(a.seed, a.t_new, node, 0);
                        uy += amp * inlet_noise<R>(a.seed, a.t_new, node, 1);
                        uz += amp * inlet_noise<R>(a.seed, a.t_new, node, 2);
                    }
                } else {
                    rho = R(a.rho_out);
                    ux = uxf;
                    uy = uyf;
                    uz = uzf;
                }
                R eb[27], ef[27];
                eq_deviation<R>(rho, Axis<R>(ux), Axis<R>(uy), Axis<R>(uz), eb);
                eq_deviation<R>(rf, Axis<R>(uxf), Axis<R>(uyf), Axis<R>(uzf), ef);
#pragma unroll
                for (int i = 0; i < 27; ++i) d[i] += eb[i] - ef[i];
            }
            T *fout = static_cast<T *>(a.fout);
            const R s = R(a.scale);
#pragma unroll
            for (int i = 0; i < 27; ++i) S::store(fout + (int64_t)i * a.stride + slot, d[i], s);
            if (a.flags & STEP_STATS) {
                const double w = (double)uz;
                a.stats[slot] += w;
                a.stats[a.stride + slot] += w * w;
            }
            if (a.flags & STEP_REDUCE) health_values(rho, ux, uy, uz, hv);
        }
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
__global__ void __launch_bounds__(STEP_THREADS) k_reduce(const void *f, const uint32_t *mask, const int2 *chunks,
                                                         const int32_t *row_base, int32_t nchunks, int64_t stride,
                                                         float inv_scale, double *partials) {
    const int gt = blockIdx.x * STEP_THREADS + threadIdx.x;
    const int chunk = gt / CHUNK;
    double hv[6] = {0, 0, 0, 0, 0, 0};
    if (chunk < nchunks) {
        const int2 ch = chunks[chunk];
        const int slot = row_base[ch.x] + ch.y + gt % CHUNK;
        if (((mask[slot] >> TYPE_SHIFT) & 3u) != TYPE_PAD) {
            double d[27], rho, ux, uy, uz;
            load_cell<P>(f, stride, slot, inv_scale, d);
            moments_of(d, rho, ux, uy, uz);
            health_values(rho, ux, uy, uz, hv);
        }
    }
    block_reduce_write(hv, partials);
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

template <int P>
cudaError_t launch_step(const StepArgs &a, bool ghost1, cudaStream_t s) {
    const int blocks = step_blocks(a.nchunks);
    if (blocks == 0) return cudaSuccess;
    if (ghost1)
        k_step<P, true><<<blocks, STEP_THREADS, 0, s>>>(a);
    else
        k_step<P, false><<<blocks, STEP_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_reduce(const void *f, const uint32_t *mask, const int2 *chunks, const int32_t *row_base,
                          int32_t nchunks, int64_t stride, float inv_scale, double *partials, cudaStream_t s) {
    const int blocks = step_blocks(nchunks);
    if (blocks == 0) return cudaSuccess;
    k_reduce<P><<<blocks, STEP_THREADS, 0, s>>>(f, mask, chunks, row_base, nchunks, stride, inv_scale, partials);
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
    template cudaError_t launch_step<P>(const StepArgs &, bool, cudaStream_t);                                     \
    template cudaError_t launch_reduce<P>(const void *, const uint32_t *, const int2 *, const int32_t *, int32_t, \
                                          int64_t, float, double *, cudaStream_t);                                 \
    template cudaError_t launch_moments<P>(const void *, const int32_t *, int64_t, int64_t, float, double *,       \
                                           cudaStream_t);                                                          \
    template cudaError_t launch_get_populations<P>(const void *, const int32_t *, int64_t, int64_t, float,         \
                                                   double *, cudaStream_t);                                        \
    template cudaError_t launch_set_populations<P>(void *, const int32_t *, int64_t, int64_t, float,               \
                                                   const double *, cudaStream_t);                                  \
    template cudaError_t launch_init_eq<P>(void *, const int32_t *, int64_t, int64_t, float, const double *,       \
                                           const double *, double, double, double, double, cudaStream_t);

}  // namespace lbm
