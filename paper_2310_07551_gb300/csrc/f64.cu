// FP64 kernels: strided batched DGEMM (mu-mode products, phi setup),
// the stencil form of the Kronecker-sum action with the reaction term, the
// pointwise stage kernels of EXPRK3DS_REAL and the phi-function evaluation.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ds_internal.h"

namespace ds {

// ---------------------------------------------------------------------------
// Strided batched GEMM (FP64, and FP32 for the CUDA-core FP32 path).
// 64x64 output tile, K chunks of 16, 256 threads,
// 4x4 outputs per thread.  GB300's FP64 pipe is narrow, so the kernel is
// built to keep it fed rather than to save bandwidth: each operand tile is
// staged once in shared memory with whichever index has unit stride mapped
// to consecutive threads.
// ---------------------------------------------------------------------------
namespace {
constexpr int BM = 64, BN = 64, BK = 16;

template <typename T, typename G>
__global__ void __launch_bounds__(256) k_gemm(G g)
{
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int b = blockIdx.z;
    const T *A = g.A + (int64_t)b * g.sAb;
    const T *B = g.B + (int64_t)b * g.sBb;
    T *C = g.C + (int64_t)b * g.sCb;
    const bool a_m_fast = (g.sAm == 1);
    const bool b_n_fast = (g.sBn == 1);

    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int e = t + 256 * r;
            int mm, kk;
            if (a_m_fast) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
            int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < g.M && gk < g.K) ? A[gm * g.sAm + gk * g.sAk] : T(0);
            int nn, kb;
            if (b_n_fast) { nn = e % BN; kb = e / BN; } else { kb = e % BK; nn = e / BK; }
            int gn = n0 + nn, gkb = k0 + kb;
            Bs[kb][nn] = (gn < g.N && gkb < g.K) ? B[gkb * g.sBk + gn * g.sBn] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty + 16 * i;
        if (gm >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int gn = n0 + tx + 16 * j;
            if (gn >= g.N) continue;
            T *c = C + gm * g.sCm + gn * g.sCn;
            T v = (T)g.alpha * acc[i][j];
            if (g.beta != 0.0) v = v + (T)g.beta * *c;
            *c = v;
        }
    }
}
}  // namespace

void launch_dgemm(const DGemm &g, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
    k_gemm<double, DGemm><<<grid, 256, 0, st>>>(g);
}

void launch_sgemm(const SGemm &g, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
    k_gemm<float, SGemm><<<grid, 256, 0, st>>>(g);
}

namespace {
// A mode product's GEMM with 64-bit sizes, launched as chunks that each fit
// the launch limits: at most 65535 batch entries (gridDim.z), 65535 row
// tiles of 64 (gridDim.y) and 2^30 columns (int indexing inside k_gemm).
// Each chunk is an independent GEMM on offset pointers, so the result is the
// same as one launch would give.
constexpr int64_t kMaxBatch = 65535, kMaxRows = 65535 * (int64_t)BM, kMaxCols = (int64_t)1 << 30;

template <typename G, typename T>
void launch_chunked(int64_t M, int64_t N, int64_t K, int64_t batch, const T *A, int64_t sAm, int64_t sAk,
                    int64_t sAb, const T *B, int64_t sBk, int64_t sBn, int64_t sBb, T *C, int64_t sCm,
                    int64_t sCn, int64_t sCb, double alpha, double beta, void (*launch)(const G &, cudaStream_t),
                    cudaStream_t st)
{
    for (int64_t b0 = 0; b0 < batch; b0 += kMaxBatch)
        for (int64_t m0 = 0; m0 < M; m0 += kMaxRows)
            for (int64_t n0 = 0; n0 < N; n0 += kMaxCols) {
                G g{};
                g.M = (int)std::min(kMaxRows, M - m0);
                g.N = (int)std::min(kMaxCols, N - n0);
                g.K = (int)K;
                g.batch = (int)std::min(kMaxBatch, batch - b0);
                g.A = A + b0 * sAb + m0 * sAm;
                g.sAm = sAm; g.sAk = sAk; g.sAb = sAb;
                g.B = B + b0 * sBb + n0 * sBn;
                g.sBk = sBk; g.sBn = sBn; g.sBb = sBb;
                g.C = C + b0 * sCb + m0 * sCm + n0 * sCn;
                g.sCm = sCm; g.sCn = sCn; g.sCb = sCb;
                g.alpha = alpha;
                g.beta = beta;
                launch(g, st);
            }
}

// Y = X x_mu L (+ beta Y) as a GEMM; L(i, j) = L[i + m j], transposed L[j + m i]
template <typename G, typename T>
void mode_product(int d, const int64_t *n, const T *X, int mu, const T *L, int transpose, T *Y, double alpha,
                  double beta, void (*launch)(const G &, cudaStream_t), cudaStream_t st)
{
    int64_t I = 1, O = 1, m = n[mu];
    for (int q = 0; q < mu; ++q) I *= n[q];
    for (int q = mu + 1; q < d; ++q) O *= n[q];
    const int64_t sLi = transpose ? m : 1, sLj = transpose ? 1 : m;
    if (mu == 0)
        // Y[r][i] = sum_j X[r][j] L(i, j): M = fibres r, N = i, K = j
        launch_chunked<G, T>(O, m, m, 1, X, m, 1, 0, L, sLj, sLi, 0, Y, m, 1, 0, alpha, beta, launch, st);
    else
        // per outer index o: Y[o][i][x] = sum_j L(i, j) X[o][j][x]
        launch_chunked<G, T>(m, I, m, O, L, sLi, sLj, 0, X, I, 1, I * m, Y, I, 1, I * m, alpha, beta, launch,
                             st);
}
}  // namespace

void launch_mode_product_f32(int d, const int64_t *n, const float *X, int mu, const float *L,
                             int transpose, float *Y, double alpha, double beta, cudaStream_t st)
{
    mode_product<SGemm, float>(d, n, X, mu, L, transpose, Y, alpha, beta, launch_sgemm, st);
}

void launch_mode_product_f64(int d, const int64_t *n, const double *X, int mu, const double *L,
                             int transpose, double *Y, double alpha, double beta, cudaStream_t st)
{
    mode_product<DGemm, double>(d, n, X, mu, L, transpose, Y, alpha, beta, launch_dgemm, st);
}

// ---------------------------------------------------------------------------
// Reaction terms (Section 3 models).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void react(const Model &m, double u, double v, double &gu, double &gv)
{
    if (m.model == DS_SCHNAKENBERG) {
        double u2v = __dmul_rn(__dmul_rn(u, u), v);
        gu = __dmul_rn(m.p[0], __dadd_rn(__dsub_rn(m.p[1], u), u2v));
        gv = __dmul_rn(m.p[0], __dsub_rn(m.p[2], u2v));
    } else if (m.model == DS_FHN) {
        gu = __dsub_rn(__dsub_rn(u, __dmul_rn(__dmul_rn(u, u), u)), v);
        gv = __dmul_rn(m.p[0], __dsub_rn(__dsub_rn(u, __dmul_rn(m.p[1], v)), m.p[2]));
    } else {
        gu = 0.0;
        gv = 0.0;
    }
}

namespace {
// K U for one point of one component: sum over modes of the tridiagonal row,
// each row summed left to right (lower, diagonal, upper), modes in order.
__device__ __forceinline__ double stencil_point(const Stencil &s, const double *U, int64_t p)
{
    double acc = 0.0;
    int64_t stride = 1, rest = p;
#pragma unroll
    for (int mu = 0; mu < kMaxD; ++mu) {
        if (mu < s.d) {
            int64_t nm = s.n[mu];
            int64_t i = rest % nm;
            rest /= nm;
            double r = __dmul_rn(s.di[mu][i], U[p]);
            if (i > 0) r = __dadd_rn(__dmul_rn(s.lo[mu][i], U[p - stride]), r);
            if (i + 1 < nm) r = __dadd_rn(r, __dmul_rn(s.up[mu][i], U[p + stride]));
            acc = __dadd_rn(acc, r);
            stride *= nm;
        }
    }
    return acc;
}

__global__ void k_rhs_f64(Stencil s0, Stencil s1, Model m, int64_t N, const double *__restrict__ U,
                          double *__restrict__ F)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        double gu, gv;
        react(m, U[p], U[N + p], gu, gv);
        F[p] = __dadd_rn(stencil_point(s0, U, p), gu);
        F[N + p] = __dadd_rn(stencil_point(s1, U + N, p), gv);
    }
}

__global__ void k_stage_diff_f64(Model m, int64_t N, const double *__restrict__ U,
                                 const double *__restrict__ a, double w1,
                                 const double *__restrict__ b, double w2, double *__restrict__ D)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        double u = U[p], v = U[N + p];
        double us = __dadd_rn(u, __dmul_rn(w1, a[p]));
        double vs = __dadd_rn(v, __dmul_rn(w1, a[N + p]));
        if (b) {
            us = __dadd_rn(us, __dmul_rn(w2, b[p]));
            vs = __dadd_rn(vs, __dmul_rn(w2, b[N + p]));
        }
        double g0u, g0v, gu, gv;
        react(m, u, v, g0u, g0v);
        react(m, us, vs, gu, gv);
        D[p] = __dsub_rn(gu, g0u);
        D[N + p] = __dsub_rn(gv, g0v);
    }
}

__global__ void k_final_f64(int64_t n2, double *__restrict__ U, const double *__restrict__ a,
                            double w1, const double *__restrict__ b, double w2)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n2;
         p += (int64_t)gridDim.x * blockDim.x)
        U[p] = __dadd_rn(__dadd_rn(U[p], __dmul_rn(w1, a[p])), __dmul_rn(w2, b[p]));
}

__global__ void k_add_g_f64(Model m, int64_t N, const double *__restrict__ U, double *__restrict__ F)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        double gu, gv;
        react(m, U[p], U[N + p], gu, gv);
        F[p] = __dadd_rn(F[p], gu);
        F[N + p] = __dadd_rn(F[N + p], gv);
    }
}

__global__ void k_nonfinite(const double *x, int64_t count, int *flag)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < count;
         p += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(x[p])) atomicExch(flag, 1);
}

// J_g(U)^T lam for one point; model as in react()
__device__ __forceinline__ void jacT(const Model &m, double u, double v, double lu, double lv, double &ou,
                                     double &ov)
{
    double juu, juv, jvu, jvv;
    if (m.model == DS_SCHNAKENBERG) {
        juu = m.p[0] * (-1.0 + 2.0 * u * v);
        juv = m.p[0] * u * u;
        jvu = -2.0 * m.p[0] * u * v;
        jvv = -m.p[0] * u * u;
    } else if (m.model == DS_FHN) {
        juu = 1.0 - 3.0 * u * u;
        juv = -1.0;
        jvu = m.p[0];
        jvv = -m.p[0] * m.p[1];
    } else {
        juu = juv = jvu = jvv = 0.0;
    }
    ou = juu * lu + jvu * lv;
    ov = juv * lu + jvv * lv;
}

// (dg/dp)(U)^T lam for one point: contributions to the three model parameters
__device__ __forceinline__ void dparam_point(const Model &m, double u, double v, double lu, double lv,
                                             double &d0, double &d1, double &d2)
{
    if (m.model == DS_SCHNAKENBERG) {
        d0 = (m.p[1] - u + u * u * v) * lu + (m.p[2] - u * u * v) * lv;
        d1 = m.p[0] * lu;
        d2 = m.p[0] * lv;
    } else if (m.model == DS_FHN) {
        d0 = (u - m.p[1] * v - m.p[2]) * lv;
        d1 = -m.p[0] * v * lv;
        d2 = -m.p[0] * lv;
    } else {
        d0 = d1 = d2 = 0.0;
    }
}

// Y = U + w1 a (+ w2 b), 2 N values
__global__ void k_axpy2(int64_t n2, const double *__restrict__ U, const double *__restrict__ a, double w1,
                        const double *__restrict__ b, double w2, double *__restrict__ Y)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n2;
         p += (int64_t)gridDim.x * blockDim.x) {
        double y = __dadd_rn(U[p], __dmul_rn(w1, a[p]));
        if (b) y = __dadd_rn(y, __dmul_rn(w2, b[p]));
        Y[p] = y;
    }
}

// D = g(Us) - g(U)
__global__ void k_gdiff(Model m, int64_t N, const double *__restrict__ U, const double *__restrict__ Us,
                        double *__restrict__ D)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        double g0u, g0v, gu, gv;
        react(m, U[p], U[N + p], g0u, g0v);
        react(m, Us[p], Us[N + p], gu, gv);
        D[p] = __dsub_rn(gu, g0u);
        D[N + p] = __dsub_rn(gv, g0v);
    }
}

// out = J_g(Us)^T lam
__global__ void k_jacT(Model m, int64_t N, const double *__restrict__ Us, const double *__restrict__ lam,
                       double *__restrict__ out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        double ou, ov;
        jacT(m, Us[p], Us[N + p], lam[p], lam[N + p], ou, ov);
        out[p] = ou;
        out[N + p] = ov;
    }
}

// K^T x for one point of one component (transposed tridiagonal rows)
__device__ __forceinline__ double stencil_point_T(const Stencil &s, const double *X, int64_t p)
{
    double acc = 0.0;
    int64_t stride = 1, rest = p;
#pragma unroll
    for (int mu = 0; mu < kMaxD; ++mu) {
        if (mu < s.d) {
            const int64_t nm = s.n[mu];
            const int64_t i = rest % nm;
            rest /= nm;
            double r = s.di[mu][i] * X[p];
            if (i > 0) r += s.up[mu][i - 1] * X[p - stride];
            if (i + 1 < nm) r += s.lo[mu][i + 1] * X[p + stride];
            acc += r;
            stride *= nm;
        }
    }
    return acc;
}

__global__ void k_kronsumT(Stencil s0, Stencil s1, int64_t N, const double *__restrict__ X,
                           double *__restrict__ Y)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        Y[p] = stencil_point_T(s0, X, p);
        Y[N + p] = stencil_point_T(s1, X + N, p);
    }
}

// lam_n = lam + lU3 + lU2 + KT + J_g(U)^T (lF - lD2 - lD3); dp += the three
// parameter gradients (block reduction, one atomic per block and parameter)
__global__ void __launch_bounds__(256) k_adjoint_final(Model m, int64_t N, const double *__restrict__ U,
                                                       const double *__restrict__ U2,
                                                       const double *__restrict__ U3,
                                                       const double *__restrict__ lam,
                                                       const double *__restrict__ lU3,
                                                       const double *__restrict__ lU2,
                                                       const double *__restrict__ KT,
                                                       const double *__restrict__ lF,
                                                       const double *__restrict__ lD2,
                                                       const double *__restrict__ lD3,
                                                       double *__restrict__ lam_n, double *dp)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double gu = lF[p] - lD2[p] - lD3[p], gv = lF[N + p] - lD2[N + p] - lD3[N + p];
        double ou, ov;
        jacT(m, U[p], U[N + p], gu, gv, ou, ov);
        lam_n[p] = lam[p] + lU3[p] + lU2[p] + KT[p] + ou;
        lam_n[N + p] = lam[N + p] + lU3[N + p] + lU2[N + p] + KT[N + p] + ov;
        if (dp) {
            double a0, a1, a2;
            dparam_point(m, U[p], U[N + p], gu, gv, a0, a1, a2);
            s0 += a0; s1 += a1; s2 += a2;
            dparam_point(m, U2[p], U2[N + p], lD2[p], lD2[N + p], a0, a1, a2);
            s0 += a0; s1 += a1; s2 += a2;
            dparam_point(m, U3[p], U3[N + p], lD3[p], lD3[N + p], a0, a1, a2);
            s0 += a0; s1 += a1; s2 += a2;
        }
    }
    if (!dp) return;
    __shared__ double red[3][256];
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) atomicAdd(dp + q, red[q][0]);
}

__global__ void __launch_bounds__(256) k_dot_accum(int64_t n, const double *__restrict__ a,
                                                   const double *__restrict__ b, double w, double *out)
{
    double s = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        s += a[p] * b[p];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, w * red[0]);
}

__global__ void __launch_bounds__(256) k_dot_kterm(Model m, int64_t N, const double *__restrict__ U,
                                                   const double *__restrict__ F,
                                                   const double *__restrict__ lF, double *out)
{
    double s0 = 0.0, s1 = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * blockDim.x) {
        double gu, gv;
        react(m, U[p], U[N + p], gu, gv);
        s0 += lF[p] * (F[p] - gu);
        s1 += lF[N + p] * (F[N + p] - gv);
    }
    __shared__ double red[2][256];
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            red[0][threadIdx.x] += red[0][threadIdx.x + k];
            red[1][threadIdx.x] += red[1][threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(out, red[0][0]);
        atomicAdd(out + 1, red[1][0]);
    }
}

int grid_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (int)std::min<int64_t>(b, 152 * 16);
}
}  // namespace

int launch_rhs_f64(const Stencil *s2, const Model &m, int64_t N, const double *U, double *F,
                   cudaStream_t st)
{
    k_rhs_f64<<<grid_for(N), 256, 0, st>>>(s2[0], s2[1], m, N, U, F);
    return 1;
}

void launch_stage_diff_f64(const Model &m, int64_t N, const double *U, const double *a, double w1,
                           const double *b, double w2, double *D, cudaStream_t st)
{
    k_stage_diff_f64<<<grid_for(N), 256, 0, st>>>(m, N, U, a, w1, b, w2, D);
}

void launch_final_f64(int64_t N, double *U, const double *a, double w1, const double *b,
                      double w2, cudaStream_t st)
{
    k_final_f64<<<grid_for(2 * N), 256, 0, st>>>(2 * N, U, a, w1, b, w2);
}

void launch_add_g_f64(const Model &m, int64_t N, const double *U, double *F, cudaStream_t st)
{
    k_add_g_f64<<<grid_for(N), 256, 0, st>>>(m, N, U, F);
}

void launch_axpy2_f64(int64_t N, const double *U, const double *a, double w1, const double *b, double w2,
                      double *Y, cudaStream_t st)
{
    k_axpy2<<<grid_for(2 * N), 256, 0, st>>>(2 * N, U, a, w1, b, w2, Y);
}
void launch_gdiff_f64(const Model &m, int64_t N, const double *U, const double *Us, double *D, cudaStream_t st)
{
    k_gdiff<<<grid_for(N), 256, 0, st>>>(m, N, U, Us, D);
}
void launch_jacT_f64(const Model &m, int64_t N, const double *Us, const double *lam, double *out,
                     cudaStream_t st)
{
    k_jacT<<<grid_for(N), 256, 0, st>>>(m, N, Us, lam, out);
}
void launch_kronsumT_f64(const Stencil *s2, int64_t N, const double *X, double *Y, cudaStream_t st)
{
    k_kronsumT<<<grid_for(N), 256, 0, st>>>(s2[0], s2[1], N, X, Y);
}
void launch_adjoint_final_f64(const Model &m, int64_t N, const double *U, const double *U2,
                              const double *U3, const double *lam, const double *lU3, const double *lU2,
                              const double *KT, const double *lF, const double *lD2, const double *lD3,
                              double *lam_n, double *dp, cudaStream_t st)
{
    k_adjoint_final<<<grid_for(N), 256, 0, st>>>(m, N, U, U2, U3, lam, lU3, lU2, KT, lF, lD2, lD3, lam_n, dp);
}

void launch_dot_accum_f64(int64_t n, const double *a, const double *b, double w, double *out,
                          cudaStream_t st)
{
    k_dot_accum<<<grid_for(n), 256, 0, st>>>(n, a, b, w, out);
}
void launch_dot_kterm_f64(const Model &m, int64_t N, const double *U, const double *F, const double *lF,
                          double *out, cudaStream_t st)
{
    k_dot_kterm<<<grid_for(N), 256, 0, st>>>(m, N, U, F, lF, out);
}

void launch_nonfinite_scan(const double *x, int64_t count, int *flag, cudaStream_t st)
{
    k_nonfinite<<<grid_for(count), 256, 0, st>>>(x, count, flag);
}

// ---------------------------------------------------------------------------
// phi_0..phi_2 of a batch of n x n matrices z_b A_b by scaling, degree-16
// Taylor and the modified squaring of Skaflestad & Wright:
//   phi_0(2Y) = phi_0(Y)^2,
//   phi_1(2Y) = (phi_0(Y) phi_1(Y) + phi_1(Y)) / 2,
//   phi_2(2Y) = (phi_0(Y) phi_2(Y) + phi_1(Y) + phi_2(Y)) / 4.
// Matrix b is squared exactly s_b times, s_b the least s >= 0 with
// ||2^-s z_b A_b||_1 <= 1/2.
// ---------------------------------------------------------------------------
namespace {
constexpr int kTaylorDeg = 16;

__global__ void k_build_X(int64_t nn, const double *const *Asrc, const double *z, double *X)
{
    const int b = blockIdx.y;
    const double *A = Asrc[b];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x)
        X[b * nn + e] = z[b] * A[e];
}

// one block per matrix: column abs-sum maximum
__global__ void k_norm1(int n, const double *X, double *out)
{
    const int b = blockIdx.x;
    const double *M = X + (int64_t)b * n * n;
    __shared__ double red[256];
    double best = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += fabs(M[i + (int64_t)n * j]);
        best = fmax(best, s);
    }
    red[threadIdx.x] = best;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = red[0];
}

__global__ void k_scale_pow2(int64_t nn, const int *s, double *X)
{
    const int b = blockIdx.y;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x)
        X[b * nn + e] = ldexp(X[b * nn + e], -s[b]);
}

__global__ void k_identity(int n, int nb, double *X)
{
    int64_t nn = (int64_t)n * n, tot = nn * nb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e % nn;
        X[e] = ((r % n) == (r / n)) ? 1.0 : 0.0;
    }
}

// phi_k += Pw / (j + k)!  for k = 0, 1, 2
__global__ void k_taylor_acc(int64_t tot, const double *Pw, double c0, double c1, double c2,
                             double *p0, double *p1, double *p2)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        double w = Pw[e];
        p0[e] = __dadd_rn(p0[e], __dmul_rn(c0, w));
        p1[e] = __dadd_rn(p1[e], __dmul_rn(c1, w));
        p2[e] = __dadd_rn(p2[e], __dmul_rn(c2, w));
    }
}

// squaring update; matrix b takes the new values only while it <= s_b
__global__ void k_square_update(int64_t nn, int it, const int *s, const double *T0,
                                const double *T1, const double *T2, double *p0, double *p1,
                                double *p2)
{
    const int b = blockIdx.y;
    if (it > s[b]) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = b * nn + e;
        double o1 = p1[q], o2 = p2[q];
        double n1 = __dmul_rn(__dadd_rn(T1[q], o1), 0.5);
        double n2 = __dmul_rn(__dadd_rn(__dadd_rn(T2[q], o1), o2), 0.25);
        p0[q] = T0[q];
        p1[q] = n1;
        p2[q] = n2;
    }
}

__global__ void k_extract(int64_t nn, const double *const *src, double *const *dst)
{
    const int b = blockIdx.y;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x)
        dst[b][e] = src[b][e];
}

// dst_b = lo_b - ell_b hi_b  (phi_{ell-1} - ell phi_ell)
__global__ void k_extract_deriv(int64_t nn, const double *const *lo, const double *const *hi,
                                const int *ell, double *const *dst)
{
    const int b = blockIdx.y;
    if (!dst[b]) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x)
        dst[b][e] = lo[b][e] - (double)ell[b] * hi[b][e];
}

void batched_square_gemm(int n, int nb, const double *A, const double *B, double *C,
                         cudaStream_t st)
{
    DGemm g{};
    int64_t nn = (int64_t)n * n;
    g.M = n; g.N = n; g.K = n; g.batch = nb;
    g.A = A; g.sAm = 1; g.sAk = n; g.sAb = nn;
    g.B = B; g.sBk = 1; g.sBn = n; g.sBb = nn;
    g.C = C; g.sCm = 1; g.sCn = n; g.sCb = nn;
    g.alpha = 1.0; g.beta = 0.0;
    launch_dgemm(g, st);
}
}  // namespace

ds_status phi_batch_f64(int n, const std::vector<PhiJob> &jobs, cudaStream_t st)
{
    const int nb = (int)jobs.size();
    if (nb == 0) return DS_OK;
    const int64_t nn = (int64_t)n * n, tot = nn * nb;
    // workspace: Y, Pw, T, phi0..2, T0..T2 (9 blocks) + tables
    double *ws = nullptr;
    DS_CUDA_TRY(cudaMallocAsync(&ws, sizeof(double) * tot * 9, st));
    double *Y = ws, *Pw = ws + tot, *T = ws + 2 * tot;
    double *p0 = ws + 3 * tot, *p1 = ws + 4 * tot, *p2 = ws + 5 * tot;
    double *T0 = ws + 6 * tot, *T1 = ws + 7 * tot, *T2 = ws + 8 * tot;

    std::vector<const double *> hA(nb);
    std::vector<double> hz(nb);
    for (int b = 0; b < nb; ++b) { hA[b] = jobs[b].A; hz[b] = jobs[b].z; }
    void *tab = nullptr;
    const size_t tab_bytes = sizeof(void *) * nb * 3 + sizeof(double) * nb * 2 + sizeof(int) * nb;
    cudaError_t e = cudaMallocAsync(&tab, tab_bytes, st);
    if (e != cudaSuccess) { cudaFreeAsync(ws, st); return fail(DS_ERR_OOM, "phi table"); }
    const double **dA = (const double **)tab;
    double **dSrc = (double **)((char *)tab + sizeof(void *) * nb);
    double **dDst = (double **)((char *)tab + sizeof(void *) * nb * 2);
    double *dz = (double *)((char *)tab + sizeof(void *) * nb * 3);
    double *dnorm = dz + nb;
    int *ds_ = (int *)(dnorm + nb);
    cudaMemcpyAsync(dA, hA.data(), sizeof(void *) * nb, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dz, hz.data(), sizeof(double) * nb, cudaMemcpyHostToDevice, st);

    dim3 g2((unsigned)std::min<int64_t>((nn + 255) / 256, 1024), nb);
    k_build_X<<<g2, 256, 0, st>>>(nn, dA, dz, Y);
    k_norm1<<<nb, 256, 0, st>>>(n, Y, dnorm);
    std::vector<double> hnorm(nb);
    cudaMemcpyAsync(hnorm.data(), dnorm, sizeof(double) * nb, cudaMemcpyDeviceToHost, st);
    DS_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int> hs(nb);
    int smax = 0;
    for (int b = 0; b < nb; ++b) {
        if (!isfinite(hnorm[b])) {
            cudaFreeAsync(ws, st); cudaFreeAsync(tab, st);
            return fail(DS_ERR_NONFINITE, "phi setup: non-finite matrix entry");
        }
        int s = 0;
        while (ldexp(hnorm[b], -s) > 0.5) ++s;
        hs[b] = s;
        smax = std::max(smax, s);
    }
    cudaMemcpyAsync(ds_, hs.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
    k_scale_pow2<<<g2, 256, 0, st>>>(nn, ds_, Y);

    // Taylor: phi_k(Y) = sum_j Y^j / (j + k)!
    double fact[kTaylorDeg + 4];
    fact[0] = 1.0;
    for (int j = 1; j < kTaylorDeg + 4; ++j) fact[j] = fact[j - 1] * j;
    const int gl = (int)std::min<int64_t>((tot + 255) / 256, 152 * 16);
    cudaMemsetAsync(p0, 0, sizeof(double) * tot * 3, st);
    k_identity<<<gl, 256, 0, st>>>(n, nb, Pw);
    for (int j = 0; j <= kTaylorDeg; ++j) {
        k_taylor_acc<<<gl, 256, 0, st>>>(tot, Pw, 1.0 / fact[j], 1.0 / fact[j + 1],
                                         1.0 / fact[j + 2], p0, p1, p2);
        if (j < kTaylorDeg) {
            batched_square_gemm(n, nb, Pw, Y, T, st);
            std::swap(Pw, T);
        }
    }
    for (int it = 1; it <= smax; ++it) {
        batched_square_gemm(n, nb, p0, p0, T0, st);
        batched_square_gemm(n, nb, p0, p1, T1, st);
        batched_square_gemm(n, nb, p0, p2, T2, st);
        k_square_update<<<g2, 256, 0, st>>>(nn, it, ds_, T0, T1, T2, p0, p1, p2);
    }
    std::vector<double *> hsrc(nb), hdst(nb);
    for (int b = 0; b < nb; ++b) {
        int l = jobs[b].ell;
        hsrc[b] = (l == 0 ? p0 : l == 1 ? p1 : p2) + b * nn;
        hdst[b] = jobs[b].out;
    }
    cudaMemcpyAsync(dSrc, hsrc.data(), sizeof(void *) * nb, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(dDst, hdst.data(), sizeof(void *) * nb, cudaMemcpyHostToDevice, st);
    k_extract<<<g2, 256, 0, st>>>(nn, (const double *const *)dSrc, (double *const *)dDst);
    bool any_d = false;
    for (int b = 0; b < nb; ++b) any_d |= (jobs[b].dout != nullptr);
    if (any_d) {
        std::vector<double *> hlo(nb), hdd(nb);
        std::vector<int> hell(nb);
        for (int b = 0; b < nb; ++b) {
            const int l = jobs[b].ell;
            hlo[b] = (l == 1 ? p0 : p1) + b * nn;
            hsrc[b] = (l == 1 ? p1 : p2) + b * nn;
            hdd[b] = jobs[b].dout;
            hell[b] = l;
        }
        // the tables are reused: dA <- lo, dSrc <- hi, dDst <- dout, ds_ <- ell
        cudaMemcpyAsync(dA, hlo.data(), sizeof(void *) * nb, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dSrc, hsrc.data(), sizeof(void *) * nb, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(dDst, hdd.data(), sizeof(void *) * nb, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(ds_, hell.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st);
        k_extract_deriv<<<g2, 256, 0, st>>>(nn, (const double *const *)dA, (const double *const *)dSrc, ds_,
                                            (double *const *)dDst);
    }
    cudaFreeAsync(ws, st);
    cudaFreeAsync(tab, st);
    DS_CUDA_TRY(cudaStreamSynchronize(st));
    DS_CUDA_TRY(cudaGetLastError());
    return DS_OK;
}

namespace {
// Aemb (2n x 2n, column-major) = [[zr A, -zi A], [zi A, zr A]]
__global__ void k_embed(int n, const double *__restrict__ A, double zr, double zi, double *__restrict__ E)
{
    const int64_t m = 2 * (int64_t)n, mm = m * m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mm;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e % m, c = e / m;
        const int64_t i = r % n, j = c % n;
        const double a = A[i + (int64_t)n * j];
        const bool lower = r >= n, right = c >= n;
        double v;
        if (lower == right) v = zr * a;        // diagonal blocks
        else if (lower) v = zi * a;            // bottom-left
        else v = -zi * a;                      // top-right
        E[e] = v;
    }
}
// re = top-left n x n block, im = bottom-left block of a 2n x 2n matrix
__global__ void k_unembed(int n, const double *__restrict__ E, double *__restrict__ re, double *__restrict__ im)
{
    const int64_t nn = (int64_t)n * n, m = 2 * (int64_t)n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        re[e] = E[i + m * j];
        im[e] = E[(i + n) + m * j];
    }
}
__global__ void k_fold_cplx(int64_t nn, const double *__restrict__ Qr, const double *__restrict__ Qi, double er,
                            double ei, double *__restrict__ M1, double *__restrict__ M2)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn;
         e += (int64_t)gridDim.x * blockDim.x) {
        M1[e] = er * Qr[e] - ei * Qi[e];
        M2[e] = -(er * Qi[e] + ei * Qr[e]);
    }
}
}  // namespace

void launch_fold_cplx(int64_t nn, const double *Qr, const double *Qi, double er, double ei, double *M1,
                      double *M2, cudaStream_t st)
{
    k_fold_cplx<<<grid_for(nn), 256, 0, st>>>(nn, Qr, Qi, er, ei, M1, M2);
}

ds_status phi_batch_cplx(int n, const std::vector<PhiJobC> &jobs, cudaStream_t st)
{
    const int nb = (int)jobs.size();
    if (nb == 0) return DS_OK;
    const int64_t m = 2 * (int64_t)n, mm = m * m;
    double *buf = nullptr;
    DS_CUDA_TRY(cudaMallocAsync(&buf, sizeof(double) * mm * nb * 2, st));
    double *emb = buf, *res = buf + mm * nb;
    std::vector<PhiJob> rj(nb);
    for (int b = 0; b < nb; ++b) {
        k_embed<<<grid_for(mm), 256, 0, st>>>(n, jobs[b].A, jobs[b].zr, jobs[b].zi, emb + b * mm);
        rj[b].A = emb + b * mm;
        rj[b].z = 1.0;
        rj[b].ell = jobs[b].ell;
        rj[b].out = res + b * mm;
        rj[b].dout = nullptr;
    }
    ds_status r = phi_batch_f64((int)m, rj, st);
    if (r != DS_OK) { cudaFreeAsync(buf, st); return r; }
    for (int b = 0; b < nb; ++b)
        k_unembed<<<grid_for((int64_t)n * n), 256, 0, st>>>(n, res + b * mm, jobs[b].out_re, jobs[b].out_im);
    cudaFreeAsync(buf, st);
    DS_CUDA_TRY(cudaStreamSynchronize(st));
    DS_CUDA_TRY(cudaGetLastError());
    return DS_OK;
}

}  // namespace ds
