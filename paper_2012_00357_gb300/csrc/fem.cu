// Constraint-set projection P_C of the DD iteration (Sec. 2, Eq. 4-6) on the
// GPU, for a box of trilinear hexahedra with 2x2x2 Gauss points, clamped at
// z = 0 and loaded by a traction on z = lz.
//
//   E = A_e{ w B^T C eps* }                       k_assemble_rhs   (Eq. 5a)
//   S = f - A_e{ w B^T sig* }                     k_assemble_rhs   (Eq. 5b)
//   K u = E,  K eta = S                           k_cg             (Eq. 5)
//   eps = B u,  sig = sig* + C B eta              k_recover        (Eq. 6)
//
// The two systems share K, so every vector stores both per node, interleaved
// as (u_x, u_y, u_z, eta_x, eta_y, eta_z): one gather of a neighbour serves
// both right-hand sides.  K is never assembled: all elements of the box have
// the same 24x24 stiffness Ke, and the node-based matrix-free product gathers
// Ke blocks over the (up to) eight elements around a node, so no atomics are
// needed and the result does not depend on scheduling.  The preconditioned CG
// runs as one cooperative persistent kernel with bounded grid barriers and
// fixed-order reductions (deterministic), warm-started from the previous DD
// iteration's (u, eta).
#include <algorithm>
#include <cmath>
#include <vector>

#include "dd_internal.cuh"
#include "fem.cuh"
#include "fem_dev.cuh"

namespace {

// ---------------------------------------------------------------------------
__global__ void k_gather_star(const int32_t *__restrict__ idx, const float *__restrict__ raw,
                              int64_t N, MetricMaps M, int64_t n_gp, double *__restrict__ star,
                              double *__restrict__ ce, unsigned *__restrict__ err) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_gp) return;
    int64_t j = idx[e];
    if (j < 0 || j >= N) {
        atomicOr(err, DEV_ERR_BOUNDS);
        j = 0;
    }
    double s[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        s[k] = (double)raw[j * 12 + k];
        star[e * 12 + k] = s[k];
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < 6; ++b) acc += M.C[6 * a + b] * s[b];
        ce[e * 6 + a] = acc;
    }
}

__global__ void k_assemble_rhs(MeshDev g, ElemOps ops, const double *__restrict__ star,
                               const double *__restrict__ ce, const double *__restrict__ f,
                               double *__restrict__ b) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= g.n_nodes) return;
    int i, j, k;
    node_ijk(g, a, i, j, k);
    double out[6] = {0, 0, 0, 0, 0, 0};
    if (k > 0 && !(g.top_fixed && k == g.nz)) {   // free node
        out[3] = f[a * 3 + 0];
        out[4] = f[a * 3 + 1];
        out[5] = f[a * 3 + 2];
        for (int oz = -1; oz <= 0; ++oz)
            for (int oy = -1; oy <= 0; ++oy)
                for (int ox = -1; ox <= 0; ++ox) {
                    int ei = i + ox, ej = j + oy, ek = k + oz;
                    if (ei < 0 || ej < 0 || ek < 0 || ei >= g.nx || ej >= g.ny || ek >= g.nz) continue;
                    int la = (-ox) + 2 * (-oy) + 4 * (-oz);
                    int64_t el = ei + (int64_t)g.nx * (ej + (int64_t)g.ny * ek);
                    for (int gp = 0; gp < 8; ++gp) {
                        int64_t e = el * 8 + gp;
                        const double *dN = ops.dN[gp][la];
                        double t[3], v[6];
#pragma unroll
                        for (int c = 0; c < 6; ++c) v[c] = ce[e * 6 + c];
                        bt_times(dN, v, t);
                        out[0] += g.w * t[0];
                        out[1] += g.w * t[1];
                        out[2] += g.w * t[2];
#pragma unroll
                        for (int c = 0; c < 6; ++c) v[c] = star[e * 12 + 6 + c];
                        bt_times(dN, v, t);
                        out[3] -= g.w * t[0];
                        out[4] -= g.w * t[1];
                        out[5] -= g.w * t[2];
                    }
                }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) b[a * 6 + c] = out[c];
}

// 3x3 block-Jacobi preconditioner: inverse of the node's diagonal block of K.
__global__ void k_block_jacobi(MeshDev g, const double *__restrict__ Ke, double *__restrict__ Minv) {
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= g.n_nodes) return;
    int i, j, k;
    node_ijk(g, a, i, j, k);
    double D[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (k > 0 && !(g.top_fixed && k == g.nz)) {   // free node
        for (int oz = -1; oz <= 0; ++oz)
            for (int oy = -1; oy <= 0; ++oy)
                for (int ox = -1; ox <= 0; ++ox) {
                    int ei = i + ox, ej = j + oy, ek = k + oz;
                    if (ei < 0 || ej < 0 || ek < 0 || ei >= g.nx || ej >= g.ny || ek >= g.nz) continue;
                    int la = (-ox) + 2 * (-oy) + 4 * (-oz);
                    for (int r = 0; r < 3; ++r)
                        for (int c = 0; c < 3; ++c) D[3 * r + c] += Ke[(3 * la + r) * 24 + 3 * la + c];
                }
        double det = D[0] * (D[4] * D[8] - D[5] * D[7]) - D[1] * (D[3] * D[8] - D[5] * D[6]) +
                     D[2] * (D[3] * D[7] - D[4] * D[6]);
        double id = 1.0 / det;
        double I[9];
        I[0] = (D[4] * D[8] - D[5] * D[7]) * id;
        I[1] = (D[2] * D[7] - D[1] * D[8]) * id;
        I[2] = (D[1] * D[5] - D[2] * D[4]) * id;
        I[3] = (D[5] * D[6] - D[3] * D[8]) * id;
        I[4] = (D[0] * D[8] - D[2] * D[6]) * id;
        I[5] = (D[2] * D[3] - D[0] * D[5]) * id;
        I[6] = (D[3] * D[7] - D[4] * D[6]) * id;
        I[7] = (D[1] * D[6] - D[0] * D[7]) * id;
        I[8] = (D[0] * D[4] - D[1] * D[3]) * id;
#pragma unroll
        for (int c = 0; c < 9; ++c) Minv[a * 9 + c] = I[c];
    } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) Minv[a * 9 + c] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// Cooperative preconditioned CG for both systems
// ---------------------------------------------------------------------------
constexpr int kCgThreads = 256;

struct CGArgs {
    MeshDev g;
    const double *Ke;      // [24 x 24]
    const double *Minv;    // [n_nodes x 9]
    const double *b;       // [n_nodes x 6]
    double *x, *r, *z, *p0, *p1, *q;
    double *part;          // [2 x grid x 8]: alternating reduction partials
    unsigned *bar;         // [2]: count, generation
    unsigned *err;
    double rtol2;
    int max_it;
    int *it_out;           // [1]
    double *res_out;       // [2] final relative residuals
};

// y_a = (K v)_a for both systems, v = vz + beta .* vp (vp may be null).
__device__ __forceinline__ void spmv_node(const MeshDev &g, const double *sKe, int64_t a,
                                          const double *vz, const double *vp, const double beta[2],
                                          double y[6]) {
    int i, j, k;
    node_ijk(g, a, i, j, k);
#pragma unroll
    for (int c = 0; c < 6; ++c) y[c] = 0.0;
    if (k == 0 || (g.top_fixed && k == g.nz)) return;   // fixed rows
    for (int oz = -1; oz <= 0; ++oz)
        for (int oy = -1; oy <= 0; ++oy)
            for (int ox = -1; ox <= 0; ++ox) {
                int ei = i + ox, ej = j + oy, ek = k + oz;
                if (ei < 0 || ej < 0 || ek < 0 || ei >= g.nx || ej >= g.ny || ek >= g.nz) continue;
                int la = (-ox) + 2 * (-oy) + 4 * (-oz);
#pragma unroll
                for (int lb = 0; lb < 8; ++lb) {
                    int64_t nb = node_id(g, ei + (lb & 1), ej + ((lb >> 1) & 1), ek + ((lb >> 2) & 1));
                    double xv[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        double t = __ldcg(vz + nb * 6 + c);
                        if (vp) t += beta[c / 3] * __ldcg(vp + nb * 6 + c);
                        xv[c] = t;
                    }
                    const double *kb = sKe + (3 * la) * 24 + 3 * lb;
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        double k0 = kb[r * 24 + 0], k1 = kb[r * 24 + 1], k2 = kb[r * 24 + 2];
                        y[r] += k0 * xv[0] + k1 * xv[1] + k2 * xv[2];
                        y[3 + r] += k0 * xv[3] + k1 * xv[4] + k2 * xv[5];
                    }
                }
            }
}

__device__ __forceinline__ void apply_minv(const double *Mi, const double *r, double *z) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            z[3 * s + a] = Mi[3 * a] * r[3 * s] + Mi[3 * a + 1] * r[3 * s + 1] + Mi[3 * a + 2] * r[3 * s + 2];
}

__global__ void __launch_bounds__(kCgThreads) k_cg(CGArgs A) {
    __shared__ double sKe[576];
    __shared__ double sh[8 * 32];
    const MeshDev &g = A.g;
    for (int t = threadIdx.x; t < 576; t += blockDim.x) sKe[t] = A.Ke[t];
    __syncthreads();
    const unsigned G = gridDim.x;
    GridBar gbar{A.bar, G, 0u};
    const int64_t stride = (int64_t)G * blockDim.x;
    const int64_t a0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double zero_beta[2] = {0.0, 0.0};
    // Phase A reduces into partA, phase B (and the set-up) into partB: a block
    // can only overwrite a buffer after every block passed the barrier that
    // follows the other buffer's reduction, i.e. after all reads of it.
    double *partA = A.part, *partB = A.part + (size_t)G * 8;

    // r = b - K x, z = M^-1 r, p0 = z; partials rz, rr, bb
    {
        double v[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t a = a0; a < g.n_nodes; a += stride) {
            double kx[6], rr[6], zz[6];
            spmv_node(g, sKe, a, A.x, nullptr, zero_beta, kx);
#pragma unroll
            for (int c = 0; c < 6; ++c) rr[c] = A.b[a * 6 + c] - kx[c];
            apply_minv(A.Minv + a * 9, rr, zz);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                A.r[a * 6 + c] = rr[c];
                A.z[a * 6 + c] = zz[c];
                A.p0[a * 6 + c] = zz[c];
                double bc = A.b[a * 6 + c];
                v[c / 3] += rr[c] * zz[c];
                v[2 + c / 3] += rr[c] * rr[c];
                v[4 + c / 3] += bc * bc;
            }
        }
        block_sum<6>(v, sh);
        if (threadIdx.x == 0)
            for (int c = 0; c < 6; ++c) partB[blockIdx.x * 8 + c] = v[c];
    }
    if (!grid_sync(gbar, A.err)) return;
    double tot[6];
    grid_total<6>(partB, G, tot, sh);
    double rz[2] = {tot[0], tot[1]}, rr[2] = {tot[2], tot[3]}, bb[2] = {tot[4], tot[5]};
    bool conv[2];
    for (int s = 0; s < 2; ++s) conv[s] = !(rr[s] > A.rtol2 * bb[s]);

    double beta[2] = {0.0, 0.0};
    double *pold = A.p0, *pnew = A.p1;
    int it = 0;
    for (; it < A.max_it && !(conv[0] && conv[1]); ++it) {
        // phase A: p_new = z + beta p_old, q = K p_new, partial p.q
        double v[2] = {0, 0};
        for (int64_t a = a0; a < g.n_nodes; a += stride) {
            double kq[6];
            spmv_node(g, sKe, a, A.z, pold, beta, kq);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                double pn = A.z[a * 6 + c] + beta[c / 3] * pold[a * 6 + c];
                pnew[a * 6 + c] = pn;
                A.q[a * 6 + c] = kq[c];
                v[c / 3] += pn * kq[c];
            }
        }
        block_sum<2>(v, sh);
        if (threadIdx.x == 0) {
            partA[blockIdx.x * 8 + 0] = v[0];
            partA[blockIdx.x * 8 + 1] = v[1];
        }
        if (!grid_sync(gbar, A.err)) return;
        double pq[2];
        grid_total<2>(partA, G, pq, sh);
        double alpha[2];
        for (int s = 0; s < 2; ++s) alpha[s] = (conv[s] || !(pq[s] > 0.0)) ? 0.0 : rz[s] / pq[s];
        // phase B: x += alpha p, r -= alpha q, z = M^-1 r, partial r.z, r.r
        double w[4] = {0, 0, 0, 0};
        for (int64_t a = a0; a < g.n_nodes; a += stride) {
            double rv[6], zv[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                double al = alpha[c / 3];
                A.x[a * 6 + c] += al * pnew[a * 6 + c];
                rv[c] = A.r[a * 6 + c] - al * A.q[a * 6 + c];
                A.r[a * 6 + c] = rv[c];
            }
            apply_minv(A.Minv + a * 9, rv, zv);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                A.z[a * 6 + c] = zv[c];
                w[c / 3] += rv[c] * zv[c];
                w[2 + c / 3] += rv[c] * rv[c];
            }
        }
        block_sum<4>(w, sh);
        if (threadIdx.x == 0)
            for (int c = 0; c < 4; ++c) partB[blockIdx.x * 8 + c] = w[c];
        if (!grid_sync(gbar, A.err)) return;
        double t4[4];
        grid_total<4>(partB, G, t4, sh);
        for (int s = 0; s < 2; ++s) {
            if (!conv[s]) {
                beta[s] = (rz[s] != 0.0) ? t4[s] / rz[s] : 0.0;
                rz[s] = t4[s];
                rr[s] = t4[2 + s];
                conv[s] = !(rr[s] > A.rtol2 * bb[s]) || !(pq[s] > 0.0);
            } else {
                beta[s] = 0.0;
            }
        }
        double *t = pold;
        pold = pnew;
        pnew = t;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *A.it_out = it;
        A.res_out[0] = bb[0] > 0 ? sqrt(rr[0] / bb[0]) : 0.0;
        A.res_out[1] = bb[1] > 0 ? sqrt(rr[1] / bb[1]) : 0.0;
    }
}

// ---------------------------------------------------------------------------
__global__ void k_recover(MeshDev g, ElemOps ops, MetricMaps M, const double *__restrict__ x,
                          const double *__restrict__ star, double *__restrict__ y,
                          double *__restrict__ dpc) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= g.n_gp) return;
    const int64_t el = e / 8;
    const int gp = (int)(e % 8);
    const int ei = (int)(el % g.nx), ej = (int)((el / g.nx) % g.ny), ek = (int)(el / ((int64_t)g.nx * g.ny));
    double eu[6] = {0, 0, 0, 0, 0, 0}, en[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        int64_t nb = node_id(g, ei + (a & 1), ej + ((a >> 1) & 1), ek + ((a >> 2) & 1));
        const double *dN = ops.dN[gp][a];
        const double *xv = x + nb * 6;
        // B_a u_a for u and for eta
        eu[0] += dN[0] * xv[0];
        eu[1] += dN[1] * xv[1];
        eu[2] += dN[2] * xv[2];
        eu[3] += dN[2] * xv[1] + dN[1] * xv[2];
        eu[4] += dN[2] * xv[0] + dN[0] * xv[2];
        eu[5] += dN[1] * xv[0] + dN[0] * xv[1];
        en[0] += dN[0] * xv[3];
        en[1] += dN[1] * xv[4];
        en[2] += dN[2] * xv[5];
        en[3] += dN[2] * xv[4] + dN[1] * xv[5];
        en[4] += dN[2] * xv[3] + dN[0] * xv[5];
        en[5] += dN[1] * xv[3] + dN[0] * xv[4];
    }
    double yy[12];
#pragma unroll
    for (int c = 0; c < 6; ++c) yy[c] = eu[c];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        double s = star[e * 12 + 6 + c];
#pragma unroll
        for (int b = 0; b < 6; ++b) s += M.C[6 * c + b] * en[b];
        yy[6 + c] = s;
    }
#pragma unroll
    for (int c = 0; c < 12; ++c) y[e * 12 + c] = yy[c];
    // distance to the current association (Eq. 3), weighted as in Eq. 2
    double de[6], ds[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        de[c] = yy[c] - star[e * 12 + c];
        ds[c] = yy[6 + c] - star[e * 12 + 6 + c];
    }
    double d = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double ce = 0.0, cs = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            ce += M.C[6 * i + k] * de[k];
            cs += M.Cinv[6 * i + k] * ds[k];
        }
        d += ce * de[i] + cs * ds[i];
    }
    dpc[e] = 0.5 * g.w * d;
}

// Iteration statistics: changed associations, sum_e 1/2 w d_e^2 after P_D,
// sum after P_C.  Every block sums a fixed share; the last block to finish
// adds the block partials in index order (deterministic for a given n).
// out: [0, 3) totals, [4] arrival counter (zero between calls), [8, 8 + 3 G)
// block partials.
constexpr int kStatsBlocks = 256;

__global__ void __launch_bounds__(256) k_iter_stats(const int32_t *__restrict__ idx_new,
                                                    const int32_t *__restrict__ idx_old,
                                                    const double *__restrict__ d2,
                                                    const double *__restrict__ dpc, int64_t n,
                                                    double w, double *__restrict__ out) {
    __shared__ double sh[3 * 32];
    __shared__ int last;
    double v[3] = {0, 0, 0};
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        v[0] += (idx_new[e] != idx_old[e]) ? 1.0 : 0.0;
        v[1] += 0.5 * w * d2[e];
        v[2] += dpc[e];
    }
    block_sum<3>(v, sh);
    double *part = out + 8;
    unsigned *cnt = reinterpret_cast<unsigned *>(out + 4);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 3; ++k) part[blockIdx.x * 3 + k] = v[k];
        __threadfence();
        last = atomicAdd(cnt, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t[3] = {0, 0, 0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        for (int k = 0; k < 3; ++k) t[k] += __ldcg(part + b * 3 + k);
    block_sum<3>(t, sh);
    if (threadIdx.x == 0) {
        out[0] = t[0];
        out[1] = t[1];
        out[2] = t[2];
        *cnt = 0u;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static const double kGP = 0.57735026918962576451;   // 1/sqrt(3)

void fem_elem_ops(const MeshDev &g, ElemOps *ops) {
    const double h[3] = {g.hx, g.hy, g.hz};
    for (int gp = 0; gp < 8; ++gp) {
        double xi[3] = {(2 * (gp & 1) - 1) * kGP, (2 * ((gp >> 1) & 1) - 1) * kGP,
                        (2 * ((gp >> 2) & 1) - 1) * kGP};
        for (int a = 0; a < 8; ++a) {
            double s[3] = {2.0 * (a & 1) - 1.0, 2.0 * ((a >> 1) & 1) - 1.0, 2.0 * ((a >> 2) & 1) - 1.0};
            double f[3] = {1 + s[0] * xi[0], 1 + s[1] * xi[1], 1 + s[2] * xi[2]};
            double d[3] = {s[0] * f[1] * f[2] / 8.0, f[0] * s[1] * f[2] / 8.0, f[0] * f[1] * s[2] / 8.0};
            for (int c = 0; c < 3; ++c) ops->dN[gp][a][c] = d[c] * 2.0 / h[c];
        }
    }
}

void fem_element_stiffness(const MeshDev &g, const ElemOps &ops, const double *C, double *Ke) {
    for (int i = 0; i < 576; ++i) Ke[i] = 0.0;
    for (int gp = 0; gp < 8; ++gp) {
        double B[6][24] = {};
        for (int a = 0; a < 8; ++a) {
            const double *d = ops.dN[gp][a];
            int c = 3 * a;
            B[0][c] = d[0];
            B[1][c + 1] = d[1];
            B[2][c + 2] = d[2];
            B[3][c + 1] = d[2];
            B[3][c + 2] = d[1];
            B[4][c] = d[2];
            B[4][c + 2] = d[0];
            B[5][c] = d[1];
            B[5][c + 1] = d[0];
        }
        double CB[6][24];
        for (int r = 0; r < 6; ++r)
            for (int c = 0; c < 24; ++c) {
                double s = 0.0;
                for (int k = 0; k < 6; ++k) s += C[6 * r + k] * B[k][c];
                CB[r][c] = s;
            }
        for (int r = 0; r < 24; ++r)
            for (int c = 0; c < 24; ++c) {
                double s = 0.0;
                for (int k = 0; k < 6; ++k) s += B[k][r] * CB[k][c];
                Ke[r * 24 + c] += g.w * s;
            }
    }
}

// The assembled K of the uniform box as a 27-point stencil of 3x3 blocks.
// The block coupling node a with its neighbour a + d is the sum of the Ke
// blocks [la, lb] over the elements that contain both nodes; which of those
// elements exist depends only on whether a lies on the low face, inside, or on
// the high face of the box along each axis.  Class c = cx + 3 cy + 9 cz with
// cx = 0 (i = 0), 1 (0 < i < nx), 2 (i = nx); offset d = (dx + 1) + 3 (dy + 1)
// + 9 (dz + 1).  Same operator as the element-by-element sum of Eq. 5, only
// the summation order differs.
void fem_stencil_table(const double *Ke, double *S) {
    for (int c = 0; c < 27; ++c) {
        const int cl[3] = {c % 3, (c / 3) % 3, c / 9};
        for (int d = 0; d < 27; ++d) {
            const int dd[3] = {d % 3 - 1, (d / 3) % 3 - 1, d / 9 - 1};
            double blk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int e = 0; e < 8; ++e) {   // bit ax of e set: the element on the low side along ax
                int la = 0, lb = 0;
                bool ok = true;
                for (int ax = 0; ax < 3 && ok; ++ax) {
                    const bool low = (e >> ax) & 1;
                    if (low ? cl[ax] == 0 : cl[ax] == 2) ok = false;   // no element there
                    const int l_a = low ? 1 : 0, l_b = l_a + dd[ax];
                    if (l_b < 0 || l_b > 1) ok = false;                // neighbour not in this element
                    la |= l_a << ax;
                    lb |= (l_b & 1) << ax;
                }
                if (!ok) continue;
                for (int r = 0; r < 3; ++r)
                    for (int k = 0; k < 3; ++k) blk[3 * r + k] += Ke[(3 * la + r) * 24 + 3 * lb + k];
            }
            for (int k = 0; k < 9; ++k) S[(c * 27 + d) * 9 + k] = blk[k];
        }
    }
}

void fem_mg_plan(const MeshDev &g, CGBuffers &cb) {
    cb.nlev = 1;
    cb.lnx[0] = g.nx;
    cb.lny[0] = g.ny;
    cb.lnz[0] = g.nz;
    cb.top = g.top_fixed;
    while (cb.nlev < kMgMaxLev) {
        const int l = cb.nlev - 1;
        if (std::min(cb.lnx[l], std::min(cb.lny[l], cb.lnz[l])) < 2) break;
        if (cb.top && cb.lnz[l] < 3) break;   // the coarser level keeps a layer of free nodes
        cb.lnx[l + 1] = (cb.lnx[l] + 1) / 2;
        cb.lny[l + 1] = (cb.lny[l] + 1) / 2;
        cb.lnz[l + 1] = (cb.lnz[l] + 1) / 2;
        cb.nlev++;
    }
    cb.glev = cb.nlev;
    cb.mg_ndof = 0;
    for (int l = 1; l < cb.nlev; ++l) {
        const int64_t dofs = 3 * (int64_t)(cb.lnx[l] + 1) * (cb.lny[l] + 1) * (cb.lnz[l] - cb.top);
        if (dofs <= kMgDirectDofs) {   // coarsest level: solved exactly
            cb.nlev = l + 1;
            cb.glev = l;
            cb.mg_ndof = (int)dofs;
            break;
        }
    }
}

void fem_mg_coarse_inverse(const CGBuffers &cb, const double *St, std::vector<float> &inv) {
    const int c = cb.glev, nx = cb.lnx[c], ny = cb.lny[c], nz = cb.lnz[c], n = cb.mg_ndof;
    const int plane = (nx + 1) * (ny + 1), zf = nz - cb.top;   // free layers 1 .. zf
    const double h = (double)(1 << c);
    std::vector<double> K((size_t)n * n, 0.0);
    for (int Z = 1; Z <= zf; ++Z)
        for (int Y = 0; Y <= ny; ++Y)
            for (int X = 0; X <= nx; ++X) {
                const int cx = X == 0 ? 0 : (X == nx ? 2 : 1), cy = Y == 0 ? 0 : (Y == ny ? 2 : 1), cz = Z == nz ? 2 : 1;
                const int cls = cx + 3 * cy + 9 * cz;
                const int fa = X + (nx + 1) * (Y + (ny + 1) * Z) - plane;
                for (int d = 0; d < 27; ++d) {
                    const int x = X + d % 3 - 1, y = Y + (d / 3) % 3 - 1, z = Z + d / 9 - 1;
                    if (x < 0 || y < 0 || z < 1 || x > nx || y > ny || z > zf) continue;
                    const int fb = x + (nx + 1) * (y + (ny + 1) * z) - plane;
                    const double *B = St + (cls * 27 + d) * 9;
                    for (int r = 0; r < 3; ++r)
                        for (int k = 0; k < 3; ++k) K[(size_t)(3 * fa + r) * n + 3 * fb + k] = h * B[3 * r + k];
                }
            }
    // Cholesky K = L L^T, then K^-1 = L^-T L^-1 (column by column)
    std::vector<double> L = K;
    for (int j = 0; j < n; ++j) {
        double d = L[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        d = std::sqrt(d);
        L[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = L[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = v / d;
        }
    }
    // columns in blocks of kB: each column takes the operations of a plain
    // column-by-column solve in the same order (so the same bits), and the
    // kB independent sums of a block keep the FMA units busy
    constexpr int kB = 32;
    std::vector<double> LT((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) LT[(size_t)i * n + k] = L[(size_t)k * n + i];
    std::vector<double> Ainv((size_t)n * n, 0.0), y((size_t)n * kB), x((size_t)n * kB);
    for (int c0 = 0; c0 < n; c0 += kB) {
        const int nb = std::min(kB, n - c0);
        for (int i = 0; i < n; ++i) {   // L y = e_col
            double v[kB];
            for (int b = 0; b < kB; ++b) v[b] = (b < nb && i == c0 + b) ? 1.0 : 0.0;
            const double *Li = &L[(size_t)i * n];
            for (int k = 0; k < i; ++k)
                for (int b = 0; b < kB; ++b) v[b] -= Li[k] * y[(size_t)k * kB + b];
            for (int b = 0; b < kB; ++b) y[(size_t)i * kB + b] = v[b] / Li[i];
        }
        for (int i = n - 1; i >= 0; --i) {   // L^T x = y
            double v[kB];
            for (int b = 0; b < kB; ++b) v[b] = y[(size_t)i * kB + b];
            const double *Ti = &LT[(size_t)i * n];
            for (int k = i + 1; k < n; ++k)
                for (int b = 0; b < kB; ++b) v[b] -= Ti[k] * x[(size_t)k * kB + b];
            for (int b = 0; b < kB; ++b) x[(size_t)i * kB + b] = v[b] / L[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i)
            for (int b = 0; b < nb; ++b) Ainv[(size_t)i * n + c0 + b] = x[(size_t)i * kB + b];
    }
    inv.assign((size_t)n * n, 0.f);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            inv[(size_t)i * n + j] = (float)(0.5 * (Ainv[(size_t)i * n + j] + Ainv[(size_t)j * n + i]));
}

double fem_jacobi_lambda_max(const double *St) {
    const int n = 6, n1 = n + 1;          // 6^3 elements, clamped at z = 0
    auto id = [&](int i, int j, int k) { return i + n1 * (j + n1 * k); };
    const int nn = n1 * n1 * n1;
    std::vector<double> x(nn * 3, 0.0), y(nn * 3, 0.0);
    uint64_t st = 0x9E3779B97F4A7C15ull;
    for (int a = n1 * n1; a < nn; ++a)
        for (int c = 0; c < 3; ++c) {
            st = st * 6364136223846793005ull + 1442695040888963407ull;
            x[a * 3 + c] = (double)(st >> 11) / 9007199254740992.0 - 0.5;
        }
    auto cls = [&](int i, int j, int k) {
        const int cx = i == 0 ? 0 : (i == n ? 2 : 1), cy = j == 0 ? 0 : (j == n ? 2 : 1), cz = k == n ? 2 : 1;
        return cx + 3 * cy + 9 * cz;
    };
    double lam = 0.0;
    for (int it = 0; it < 120; ++it) {
        double nx2 = 0.0, ny2 = 0.0;
        for (int k = 1; k <= n; ++k)
            for (int j = 0; j <= n; ++j)
                for (int i = 0; i <= n; ++i) {
                    const int c = cls(i, j, k);
                    double kx[3] = {0, 0, 0};
                    for (int d = 0; d < 27; ++d) {
                        const int I = i + d % 3 - 1, J = j + (d / 3) % 3 - 1, K = k + d / 9 - 1;
                        if (I < 0 || J < 0 || K < 1 || I > n || J > n || K > n) continue;
                        const double *B = St + (c * 27 + d) * 9;
                        const double *v = &x[id(I, J, K) * 3];
                        for (int r = 0; r < 3; ++r) kx[r] += B[3 * r] * v[0] + B[3 * r + 1] * v[1] + B[3 * r + 2] * v[2];
                    }
                    // solve D y = K x with the node's diagonal block
                    const double *D = St + (c * 27 + 13) * 9;
                    const double det = D[0] * (D[4] * D[8] - D[5] * D[7]) - D[1] * (D[3] * D[8] - D[5] * D[6]) +
                                       D[2] * (D[3] * D[7] - D[4] * D[6]);
                    const double I9[9] = {(D[4] * D[8] - D[5] * D[7]) / det, (D[2] * D[7] - D[1] * D[8]) / det,
                                          (D[1] * D[5] - D[2] * D[4]) / det, (D[5] * D[6] - D[3] * D[8]) / det,
                                          (D[0] * D[8] - D[2] * D[6]) / det, (D[2] * D[3] - D[0] * D[5]) / det,
                                          (D[3] * D[7] - D[4] * D[6]) / det, (D[1] * D[6] - D[0] * D[7]) / det,
                                          (D[0] * D[4] - D[1] * D[3]) / det};
                    double *o = &y[id(i, j, k) * 3];
                    for (int r = 0; r < 3; ++r) o[r] = I9[3 * r] * kx[0] + I9[3 * r + 1] * kx[1] + I9[3 * r + 2] * kx[2];
                }
        for (int a = 0; a < nn * 3; ++a) {
            nx2 += x[a] * x[a];
            ny2 += y[a] * y[a];
        }
        lam = std::sqrt(ny2 / nx2);
        const double s = 1.0 / std::sqrt(ny2);
        for (int a = 0; a < nn * 3; ++a) x[a] = y[a] * s;
    }
    return lam;
}

void fem_top_rotation(const MeshDev &g, double theta, double lx, double ly, double *x) {
    const double c = std::cos(theta), s = std::sin(theta);
    for (int j = 0; j <= g.ny; ++j)
        for (int i = 0; i <= g.nx; ++i) {
            const double dx = i * g.hx - 0.5 * lx, dy = j * g.hy - 0.5 * ly;
            double *u = x + (size_t)(i + (int64_t)(g.nx + 1) * (j + (int64_t)(g.ny + 1) * g.nz)) * 6;
            u[0] = (c - 1.0) * dx - s * dy;
            u[1] = s * dx + (c - 1.0) * dy;
            u[2] = 0.0;
        }
}

void fem_traction_force(const MeshDev &g, const dd_load &L, double lx, double ly, double *f) {
    for (int64_t i = 0; i < g.n_nodes * 3; ++i) f[i] = 0.0;
    const double hx = g.hx, hy = g.hy, wq = hx * hy / 4.0;
    for (int i = 0; i < g.nx; ++i)
        for (int j = 0; j < g.ny; ++j)
            for (int qx = 0; qx < 2; ++qx)
                for (int qy = 0; qy < 2; ++qy) {
                    double gx = (2 * qx - 1) * kGP, gy = (2 * qy - 1) * kGP;
                    double x = (i + 0.5 * (1 + gx)) * hx, y = (j + 0.5 * (1 + gy)) * hy;
                    double t[3];
                    for (int c = 0; c < 3; ++c) t[c] = L.t0[c] + L.tx[c] * (x - lx / 2) + L.ty[c] * (y - ly / 2);
                    for (int ax = 0; ax < 2; ++ax)
                        for (int ay = 0; ay < 2; ++ay) {
                            double N = 0.25 * (1 + (2 * ax - 1) * gx) * (1 + (2 * ay - 1) * gy);
                            int64_t n = (i + ax) + (int64_t)(g.nx + 1) * ((j + ay) + (int64_t)(g.ny + 1) * g.nz);
                            for (int c = 0; c < 3; ++c) f[n * 3 + c] += N * t[c] * wq;
                        }
                }
}

dd_status fem_gather_star(dd_dataset *ds, const int32_t *idx, int64_t n_gp, double *star, double *ce,
                          cudaStream_t s) {
    ds->ctx->launches++;
    k_gather_star<<<(unsigned)((n_gp + 255) / 256), 256, 0, s>>>(idx, ds->raw, ds->N, ds->M, n_gp, star,
                                                                ce, ds->ctx->dev_err);
    DD_TRY_CUDA(ds->ctx, cudaGetLastError());
    return DD_OK;
}

dd_status fem_assemble_rhs(dd_ctx *ctx, const MeshDev &g, const ElemOps &ops, const double *star,
                           const double *ce, const double *f, double *b, cudaStream_t s) {
    ctx->launches++;
    k_assemble_rhs<<<(unsigned)((g.n_nodes + 127) / 128), 128, 0, s>>>(g, ops, star, ce, f, b);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

dd_status fem_block_jacobi(dd_ctx *ctx, const MeshDev &g, const double *Ke, double *Minv, cudaStream_t s) {
    ctx->launches++;
    k_block_jacobi<<<(unsigned)((g.n_nodes + 127) / 128), 128, 0, s>>>(g, Ke, Minv);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

// Mixed-precision CG (FP32 Krylov iterations inside FP64 iterative
// refinement, batch.cu) of one system.
dd_status fem_cg_mixed(dd_ctx *ctx, const MeshDev &g, const CGBuffers &B, double rtol, int max_it,
                       cudaStream_t s) {
    const MeshDev *gs[1] = {&g};
    const CGBuffers *cbs[1] = {&B};
    int *it_dev = nullptr;
    DD_TRY(dd_cg_segments(ctx, gs, cbs, 1, rtol, max_it, s, &it_dev));
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(B.it_out, it_dev, sizeof(int), cudaMemcpyDeviceToDevice, s));
    return DD_OK;
}

dd_status fem_cg(dd_ctx *ctx, const MeshDev &g, const CGBuffers &B, double rtol, int max_it,
                 cudaStream_t s) {
    int occ = 0;
    DD_TRY_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg, kCgThreads, 0));
    if (occ < 1) return dd_fail(ctx, DD_ERR_CUDA, "CG kernel cannot be resident");
    int64_t want = (g.n_nodes + kCgThreads - 1) / kCgThreads;
    int grid = (int)std::min<int64_t>(want, (int64_t)occ * ctx->n_sm);
    grid = std::max(grid, 1);
    CGArgs A;
    A.g = g;
    A.Ke = B.Ke;
    A.Minv = B.Minv;
    A.b = B.b;
    A.x = B.x;
    A.r = B.r;
    A.z = B.z;
    A.p0 = B.p0;
    A.p1 = B.p1;
    A.q = B.q;
    A.part = B.part;
    A.bar = B.bar;
    A.err = ctx->dev_err;
    A.rtol2 = rtol * rtol;
    A.max_it = max_it;
    A.it_out = B.it_out;
    A.res_out = B.res_out;
    DD_TRY_CUDA(ctx, cudaMemsetAsync(B.bar, 0, 2 * sizeof(unsigned), s));
    void *args[] = {&A};
    ctx->launches++;
    DD_TRY_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)k_cg, dim3(grid), dim3(kCgThreads), args, 0, s));
    return DD_OK;
}

dd_status fem_recover(dd_dataset *ds, const MeshDev &g, const ElemOps &ops, const double *x,
                      const double *star, double *y, double *dpc, cudaStream_t s) {
    ds->ctx->launches++;
    k_recover<<<(unsigned)((g.n_gp + 127) / 128), 128, 0, s>>>(g, ops, ds->M, x, star, y, dpc);
    DD_TRY_CUDA(ds->ctx, cudaGetLastError());
    return DD_OK;
}

dd_status fem_iter_stats(dd_ctx *ctx, const int32_t *idx_new, const int32_t *idx_old, const double *d2,
                         const double *dpc, int64_t n, double w, double *out, cudaStream_t s) {
    ctx->launches++;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(kStatsBlocks, (n + 1023) / 1024));
    k_iter_stats<<<grid, 256, 0, s>>>(idx_new, idx_old, d2, dpc, n, w, out);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}
