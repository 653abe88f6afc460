// Kernels of the reverse sweep (gradient of a field-level loss with respect to the
// initial white noise) through the FP32 particle-mesh step.
//
// Positions enter as uint32 ticks and derivatives are taken with respect to the box
// fraction u = ticks / 2^32.  With mesh coordinate s = u n - 1/2 the CIC weights of a
// particle along one axis are (1 - d, d), d = s - floor(s), so dW/du = n (-1, +1) on
// the same side of a cell boundary as the forward floor().
#include "internal.h"
#include "particles.h"

namespace pm {

namespace {

struct Cic1 {
    int i0, i1;
    float w1;
};
__device__ __forceinline__ Cic1 decode(uint32_t u, int logn, float inv_cell_ticks) {
    const int sh = 32 - logn;
    const uint32_t t = u - (1u << (sh - 1));
    Cic1 c;
    c.i0 = (int)(t >> sh);
    c.i1 = (c.i0 + 1) & ((1 << logn) - 1);
    c.w1 = __uint2float_rn(t & ((1u << sh) - 1u)) * inv_cell_ticks;
    return c;
}

// grad_u of sum_c F(c) W(u, c) for the three axes.
__device__ __forceinline__ void grad_gather(const float* __restrict__ F, size_t n, const Cic1& cx, const Cic1& cy,
                                            const Cic1& cz, float out[3]) {
    const float nf = (float)n;
    const int ix[2] = {cx.i0, cx.i1}, iy[2] = {cy.i0, cy.i1}, iz[2] = {cz.i0, cz.i1};
    const float wx[2] = {1.0f - cx.w1, cx.w1}, wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
    const float dw[2] = {-nf, nf};
    out[0] = out[1] = out[2] = 0.0f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float f = __ldg(F + ((size_t)ix[a] * n + iy[b]) * n + iz[c]);
                out[0] += dw[a] * wy[b] * wz[c] * f;
                out[1] += wx[a] * dw[b] * wz[c] * f;
                out[2] += wx[a] * wy[b] * dw[c] * f;
            }
}

}  // namespace

// lam_u (+)= scale grad_u interp(F)
__global__ void k_adj_gather(const uint32_t* __restrict__ x, int64_t count, int logn, float inv_cell_ticks,
                             const float* __restrict__ F, float scale, int accumulate, float* __restrict__ lam_u) {
    const size_t n = (size_t)1 << logn;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const Cic1 cx = decode(x[i], logn, inv_cell_ticks), cy = decode(x[count + i], logn, inv_cell_ticks),
                   cz = decode(x[2 * count + i], logn, inv_cell_ticks);
        float g[3];
        grad_gather(F, n, cx, cy, cz, g);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float v = scale * g[j];
            lam_u[j * count + i] = accumulate ? lam_u[j * count + i] + v : v;
        }
    }
}

// lam_u += K sum_j v_j grad_u interp(G_j)  (the direct part of the transposed kick)
__global__ void k_adj_direct(const uint32_t* __restrict__ x, int64_t count, int logn, float inv_cell_ticks,
                             const float* __restrict__ v, const float* __restrict__ G0, const float* __restrict__ G1,
                             const float* __restrict__ G2, float K, float* __restrict__ lam_u) {
    const size_t n = (size_t)1 << logn;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const Cic1 cx = decode(x[i], logn, inv_cell_ticks), cy = decode(x[count + i], logn, inv_cell_ticks),
                   cz = decode(x[2 * count + i], logn, inv_cell_ticks);
        const float v0 = v[i], v1 = v[count + i], v2 = v[2 * count + i];
        float g0[3], g1[3], g2[3];
        grad_gather(G0, n, cx, cy, cz, g0);
        grad_gather(G1, n, cx, cy, cz, g1);
        grad_gather(G2, n, cx, cy, cz, g2);
#pragma unroll
        for (int j = 0; j < 3; ++j) lam_u[j * count + i] += K * (v0 * g0[j] + v1 * g1[j] + v2 * g2[j]);
    }
}

// The particle side of the transposed kick at positions x (one pass, the next particle's
// inputs loaded one iteration ahead):
//   lam_u += K sum_j v_j grad_u interp(G_j) + K mass grad_u interp(rho_bar)
// followed, when drift_next != 0, by the transposed drift of the step before,
//   v += drift_next lam_u   (v = lam_p, updated in place).
__global__ void __launch_bounds__(256) k_adj_kick(const uint32_t* __restrict__ x, int64_t count, int logn,
                                                  float inv_cell_ticks, float* __restrict__ v,
                                                  const float* __restrict__ G0, const float* __restrict__ G1,
                                                  const float* __restrict__ G2, const float* __restrict__ rho_bar,
                                                  float K, float Km, float drift_next, float* __restrict__ lam_u) {
    const float nf = (float)(1 << logn);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t nx0 = 0, nx1 = 0, nx2 = 0;
    float nv0 = 0.f, nv1 = 0.f, nv2 = 0.f;
    if (i < count) {
        nx0 = x[i], nx1 = x[count + i], nx2 = x[2 * count + i];
        nv0 = v[i], nv1 = v[count + i], nv2 = v[2 * count + i];
    }
    for (; i < count; i += stride) {
        const uint32_t u0 = nx0, u1 = nx1, u2 = nx2;
        const float v0 = nv0, v1 = nv1, v2 = nv2;
        if (i + stride < count) {
            const int64_t j = i + stride;
            nx0 = x[j], nx1 = x[count + j], nx2 = x[2 * count + j];
            nv0 = v[j], nv1 = v[count + j], nv2 = v[2 * count + j];
        }
        const Cic1 cx = decode(u0, logn, inv_cell_ticks), cy = decode(u1, logn, inv_cell_ticks),
                   cz = decode(u2, logn, inv_cell_ticks);
        const uint32_t ix[2] = {(uint32_t)cx.i0, (uint32_t)cx.i1}, iy[2] = {(uint32_t)cy.i0, (uint32_t)cy.i1},
                       iz[2] = {(uint32_t)cz.i0, (uint32_t)cz.i1};
        const float wx[2] = {1.0f - cx.w1, cx.w1}, wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
        const float dw[2] = {-nf, nf};
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const uint32_t o = (((ix[a] << logn) + iy[b]) << logn) + iz[c];
                    // K sum_j v_j G_j + K mass rho_bar at the corner
                    const float s = K * (v0 * __ldg(G0 + o) + v1 * __ldg(G1 + o) + v2 * __ldg(G2 + o)) +
                                    Km * __ldg(rho_bar + o);
                    g0 = fmaf(dw[a] * wy[b] * wz[c], s, g0);
                    g1 = fmaf(wx[a] * dw[b] * wz[c], s, g1);
                    g2 = fmaf(wx[a] * wy[b] * dw[c], s, g2);
                }
        const float l0 = lam_u[i] + g0, l1 = lam_u[count + i] + g1, l2 = lam_u[2 * count + i] + g2;
        lam_u[i] = l0;
        lam_u[count + i] = l1;
        lam_u[2 * count + i] = l2;
        if (drift_next != 0.f) {
            v[i] = fmaf(drift_next, l0, v0);
            v[count + i] = fmaf(drift_next, l1, v1);
            v[2 * count + i] = fmaf(drift_next, l2, v2);
        }
    }
}

// First-order gradient (g = -grad of the CIC interpolant of phi, the update's fd1_force):
// V(c) += -sum_p sum_j v_j dW(u_p, c)/dx_j with dW/dx_j = inv_d (-1, +1) along j times the other
// two weights (x in Mpc/h, inv_d = n / L): the transposed gradient gather, one scalar mesh.
__global__ void k_deposit_grad(const uint32_t* __restrict__ x, int64_t count, int logn, float inv_cell_ticks,
                               const float* __restrict__ v, float inv_d, float* __restrict__ V) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const Cic1 cx = decode(x[i], logn, inv_cell_ticks), cy = decode(x[count + i], logn, inv_cell_ticks),
                   cz = decode(x[2 * count + i], logn, inv_cell_ticks);
        const float v0 = -inv_d * v[i], v1 = -inv_d * v[count + i], v2 = -inv_d * v[2 * count + i];
        const uint32_t ix[2] = {(uint32_t)cx.i0, (uint32_t)cx.i1}, iy[2] = {(uint32_t)cy.i0, (uint32_t)cy.i1},
                       iz[2] = {(uint32_t)cz.i0, (uint32_t)cz.i1};
        const float wx[2] = {1.0f - cx.w1, cx.w1}, wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
        const float sg[2] = {-1.0f, 1.0f};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float w = v0 * sg[a] * wy[b] * wz[c] + v1 * wx[a] * sg[b] * wz[c] + v2 * wx[a] * wy[b] * sg[c];
                    atomicAdd(V + (((ix[a] << logn) + iy[b]) << logn) + iz[c], w);
                }
    }
}

// The particle side of the first-order gradient's transposed kick:
//   lam_u_i += K sum_j v_j d/du_i g_j(u) + Km grad_u interp(rho_bar),
// g_j = -sum_c dW/dx_j phi(c), whose u_i derivative keeps only the mixed (i != j) terms of the
// trilinear weight; then the transposed drift v += drift_next lam_u as in k_adj_kick.
__global__ void __launch_bounds__(256) k_adj_kick_fd(const uint32_t* __restrict__ x, int64_t count, int logn,
                                                     float inv_cell_ticks, float* __restrict__ v,
                                                     const float* __restrict__ phi, const float* __restrict__ rho_bar,
                                                     float K, float Km, float inv_d, float drift_next,
                                                     float* __restrict__ lam_u) {
    const float nf = (float)(1 << logn);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float v0 = v[i], v1 = v[count + i], v2 = v[2 * count + i];
        const Cic1 cx = decode(x[i], logn, inv_cell_ticks), cy = decode(x[count + i], logn, inv_cell_ticks),
                   cz = decode(x[2 * count + i], logn, inv_cell_ticks);
        const uint32_t ix[2] = {(uint32_t)cx.i0, (uint32_t)cx.i1}, iy[2] = {(uint32_t)cy.i0, (uint32_t)cy.i1},
                       iz[2] = {(uint32_t)cz.i0, (uint32_t)cz.i1};
        const float wx[2] = {1.0f - cx.w1, cx.w1}, wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
        const float sg[2] = {-1.0f, 1.0f};
        const float Kd = -K * inv_d * nf;  // -K (d w/dx) (d w/du) per pair of signs
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const uint32_t o = (((ix[a] << logn) + iy[b]) << logn) + iz[c];
                    const float f = __ldg(phi + o), r = Km * nf * __ldg(rho_bar + o);
                    const float sx = sg[a], sy = sg[b], sz = sg[c];
                    g0 += sx * (Kd * (v1 * sy * wz[c] + v2 * sz * wy[b]) * f + r * wy[b] * wz[c]);
                    g1 += sy * (Kd * (v0 * sx * wz[c] + v2 * sz * wx[a]) * f + r * wx[a] * wz[c]);
                    g2 += sz * (Kd * (v0 * sx * wy[b] + v1 * sy * wx[a]) * f + r * wx[a] * wy[b]);
                }
        const float l0 = lam_u[i] + g0, l1 = lam_u[count + i] + g1, l2 = lam_u[2 * count + i] + g2;
        lam_u[i] = l0;
        lam_u[count + i] = l1;
        lam_u[2 * count + i] = l2;
        if (drift_next != 0.f) {
            v[i] = fmaf(drift_next, l0, v0);
            v[count + i] = fmaf(drift_next, l1, v1);
            v[2 * count + i] = fmaf(drift_next, l2, v2);
        }
    }
}

// V_j(c) += sum_p v_j W(u_p, c) for the three components, particles in lattice order
// (id = (ix np + iy) np + iz) walked along x in runs of RUN (thread = (iz, iy, run); the
// next particle is loaded one iteration ahead).  With MERGE (lattice as fine as the mesh)
// the next particle along x usually starts one cell further in x, so its lower-x corners
// are the current upper-x corners: those 12 weighted values are carried in registers and
// added with the next particle's (12 atomics a particle instead of 24).
template <bool MERGE>
__global__ void __launch_bounds__(256) k_deposit_vec_rows(const uint32_t* __restrict__ x, int lognp, int logn,
                                                          int run, float inv_cell_ticks, const float* __restrict__ v,
                                                          float* __restrict__ V0, float* __restrict__ V1,
                                                          float* __restrict__ V2) {
    const int np = 1 << lognp;
    const int64_t count = (int64_t)1 << (3 * lognp);
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lz = (int)(gid & (np - 1)), ly = (int)((gid >> lognp) & (np - 1));
    const int lx0 = (int)(gid >> (2 * lognp)) * run;
    if (lx0 >= np) return;
    const int64_t xstride = (int64_t)1 << (2 * lognp);
    const int64_t id0 = (((int64_t)lx0 << lognp) + ly) * np + lz;
    uint32_t nu0 = x[id0], nu1 = x[count + id0], nu2 = x[2 * count + id0];
    float nv0 = v[id0], nv1 = v[count + id0], nv2 = v[2 * count + id0];
    uint32_t carry_cell = 0xffffffffu, carry_o[4] = {0u, 0u, 0u, 0u};
    float carry[4][3];
    auto add3 = [&](uint32_t o, float a, float b, float c) {
        atomicAdd(V0 + o, a);
        atomicAdd(V1 + o, b);
        atomicAdd(V2 + o, c);
    };
#pragma unroll 1
    for (int k = 0; k < run; ++k) {
        const int64_t id = id0 + k * xstride;
        const uint32_t u0 = nu0, u1 = nu1, u2 = nu2;
        const float v0 = nv0, v1 = nv1, v2 = nv2;
        if (k + 1 < run) {
            const int64_t j = id + xstride;
            nu0 = x[j], nu1 = x[count + j], nu2 = x[2 * count + j];
            nv0 = v[j], nv1 = v[count + j], nv2 = v[2 * count + j];
        }
        const Cic1 cx = decode(u0, logn, inv_cell_ticks), cy = decode(u1, logn, inv_cell_ticks),
                   cz = decode(u2, logn, inv_cell_ticks);
        const uint32_t iy[2] = {(uint32_t)cy.i0, (uint32_t)cy.i1}, iz[2] = {(uint32_t)cz.i0, (uint32_t)cz.i1};
        const float wx0 = 1.0f - cx.w1, wx1 = cx.w1;
        const float wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
        const uint32_t cell = ((((uint32_t)cx.i0 << logn) | iy[0]) << logn) | iz[0];
        const bool merge = MERGE && cell == carry_cell;
        if (MERGE && !merge && carry_cell != 0xffffffffu) {
#pragma unroll
            for (int q = 0; q < 4; ++q) add3(carry_o[q], carry[q][0], carry[q][1], carry[q][2]);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int q = 2 * b + c;
                const float w = wy[b] * wz[c];
                const uint32_t o0 = ((((uint32_t)cx.i0 << logn) + iy[b]) << logn) + iz[c];
                const uint32_t o1 = ((((uint32_t)cx.i1 << logn) + iy[b]) << logn) + iz[c];
                float a0 = wx0 * w * v0, a1 = wx0 * w * v1, a2 = wx0 * w * v2;
                if (merge) {
                    a0 += carry[q][0];
                    a1 += carry[q][1];
                    a2 += carry[q][2];
                }
                add3(o0, a0, a1, a2);
                if (MERGE) {
                    carry[q][0] = wx1 * w * v0;
                    carry[q][1] = wx1 * w * v1;
                    carry[q][2] = wx1 * w * v2;
                    carry_o[q] = o1;
                } else {
                    add3(o1, wx1 * w * v0, wx1 * w * v1, wx1 * w * v2);
                }
            }
        if (MERGE) carry_cell = ((((uint32_t)cx.i1 << logn) | iy[0]) << logn) | iz[0];
    }
    if (MERGE && carry_cell != 0xffffffffu) {
#pragma unroll
        for (int q = 0; q < 4; ++q) add3(carry_o[q], carry[q][0], carry[q][1], carry[q][2]);
    }
}

// out = sum_j i k_j c(k) in_j on the [kz][kx][ky] half spectrum, with
//   mode 0 (transposed force): c = -(3/2) Om / (k^2 n^3), k_j = 0 at the Nyquist index;
//   mode 1 (transposed Zel'dovich map): c = -amp(|n|^2) np^{-3/2} / k^2, zero on every
//   mode with a Nyquist component.  The zero mode is zero.
__global__ void k_adj_combine(const float2* __restrict__ in0, const float2* __restrict__ in1,
                              const float2* __restrict__ in2, float2* __restrict__ out, int n, double kf, double coef,
                              const double* __restrict__ amp, int mode) {
    const int M = n / 2;
    const int64_t total = (int64_t)(M + 1) * n * n;
    const float kff = (float)kf, kf2 = kff * kff, coef_f = (float)coef;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int kz = (int)(e / ((int64_t)n * n));
        const int rem = (int)(e - (int64_t)kz * n * n);
        const int nx = signed_k(rem / n, n), ny = signed_k(rem % n, n), nz = kz;
        const int n2 = nx * nx + ny * ny + nz * nz;
        float2 r = make_float2(0.f, 0.f);
        const bool nyq_any = (2 * nx == -n) || (2 * ny == -n) || (nz == M);
        if (n2 > 0 && !(mode == 1 && nyq_any)) {
            // FP32 arithmetic (no FP64 divide per mode): c = coef / (kf^2 n2) [* amp(n2)]
            float c = coef_f / (kf2 * (float)n2);
            if (mode == 1) c *= (float)amp[n2];
            const float kx = (2 * nx == -n) ? 0.f : kff * (float)nx;
            const float ky = (2 * ny == -n) ? 0.f : kff * (float)ny;
            const float kzz = (nz == M) ? 0.f : kff * (float)nz;
            const float2 a = in0[e], b = in1[e], d = in2[e];
            // i k_j c z = c k_j (-z.y, z.x)
            const float sx = kx * a.x + ky * b.x + kzz * d.x;
            const float sy = kx * a.y + ky * b.y + kzz * d.y;
            r = make_float2(-c * sy, c * sx);
        }
        out[e] = r;
    }
}

// lambda_rho = 2 (delta - target) / n^3 (in place over delta) and sum (delta - target)^2
__global__ void k_loss(float* __restrict__ delta, const float* __restrict__ target, int64_t n3, double inv_n3,
                       double* __restrict__ acc) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = delta[i] - target[i];
        s += (double)d * (double)d;
        delta[i] = (float)(2.0 * inv_n3 * (double)d);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

// y = alpha a + beta b (three components, count each); b may be null
__global__ void k_axpby(float* __restrict__ y, const float* __restrict__ a, const float* __restrict__ b, int64_t m,
                        float alpha, float beta) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = alpha * a[i] + (b ? beta * b[i] : 0.0f);
}

static unsigned blocks_for(int64_t count) {
    int64_t b = (count + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t adj_gather(const uint32_t* x, int64_t count, int n, const float* F, float scale, int accumulate,
                       float* lam_u, cudaStream_t st) {
    const int logn = ilog2(n);
    k_adj_gather<<<blocks_for(count), 256, 0, st>>>(x, count, logn, (float)ldexp(1.0, -(32 - logn)), F, scale,
                                                    accumulate, lam_u);
    return cudaGetLastError();
}

cudaError_t adj_direct(const uint32_t* x, int64_t count, int n, const float* v, const float* const* G, float K,
                       float* lam_u, cudaStream_t st) {
    const int logn = ilog2(n);
    k_adj_direct<<<blocks_for(count), 256, 0, st>>>(x, count, logn, (float)ldexp(1.0, -(32 - logn)), v, G[0], G[1],
                                                    G[2], K, lam_u);
    return cudaGetLastError();
}

cudaError_t adj_kick_particles(const uint32_t* x, int64_t count, int n, float* v, const float* const* G,
                               const float* rho_bar, float K, float Km, float drift_next, float* lam_u,
                               cudaStream_t st) {
    const int logn = ilog2(n);
    k_adj_kick<<<blocks_for(count), 256, 0, st>>>(x, count, logn, (float)ldexp(1.0, -(32 - logn)), v, G[0], G[1], G[2],
                                                  rho_bar, K, Km, drift_next, lam_u);
    return cudaGetLastError();
}

cudaError_t deposit_grad(const uint32_t* x, int64_t count, int n, const float* v, double inv_d, float* V,
                         cudaStream_t st) {
    const int logn = ilog2(n);
    k_deposit_grad<<<blocks_for(count), 256, 0, st>>>(x, count, logn, (float)ldexp(1.0, -(32 - logn)), v, (float)inv_d,
                                                      V);
    return cudaGetLastError();
}

cudaError_t adj_kick_particles_fd(const uint32_t* x, int64_t count, int n, float* v, const float* phi,
                                  const float* rho_bar, float K, float Km, double inv_d, float drift_next, float* lam_u,
                                  cudaStream_t st) {
    const int logn = ilog2(n);
    k_adj_kick_fd<<<blocks_for(count), 256, 0, st>>>(x, count, logn, (float)ldexp(1.0, -(32 - logn)), v, phi, rho_bar,
                                                     K, Km, (float)inv_d, drift_next, lam_u);
    return cudaGetLastError();
}

cudaError_t deposit_vec(const uint32_t* x, int np, int n, const float* v, float* const* V, cudaStream_t st) {
    const int lognp = ilog2(np), logn = ilog2(n);
    // rows of `run` particles a thread: long rows share more corners, short rows give more
    // threads; about two waves of full occupancy when the lattice is small
    int run = 4;
    while (run < 16 && (int64_t)np * np * np / run > 2 * 152 * 2048) run *= 2;
    if (run > np) run = np;
    const int64_t threads = (int64_t)np * np * (np / run);
    const unsigned blocks = (unsigned)((threads + 255) / 256);
    const float inv = (float)ldexp(1.0, -(32 - logn));
    if (n == np)
        k_deposit_vec_rows<true><<<blocks, 256, 0, st>>>(x, lognp, logn, run, inv, v, V[0], V[1], V[2]);
    else
        k_deposit_vec_rows<false><<<blocks, 256, 0, st>>>(x, lognp, logn, run, inv, v, V[0], V[1], V[2]);
    return cudaGetLastError();
}

cudaError_t adj_combine(const float2* const* in, float2* out, int n, double kf, double coef, const double* amp,
                        int mode, cudaStream_t st) {
    const int64_t total = (int64_t)(n / 2 + 1) * n * n;
    k_adj_combine<<<blocks_for(total), 256, 0, st>>>(in[0], in[1], in[2], out, n, kf, coef, amp, mode);
    return cudaGetLastError();
}

cudaError_t loss_mse(float* delta, const float* target, int64_t n3, double* acc, cudaStream_t st) {
    k_loss<<<blocks_for(n3), 256, 0, st>>>(delta, target, n3, 1.0 / (double)n3, acc);
    return cudaGetLastError();
}

cudaError_t axpby(float* y, const float* a, const float* b, int64_t m, float alpha, float beta, cudaStream_t st) {
    k_axpby<<<blocks_for(m), 256, 0, st>>>(y, a, b, m, alpha, beta);
    return cudaGetLastError();
}

}  // namespace pm
