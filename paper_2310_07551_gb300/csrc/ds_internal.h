// Internal declarations of the ds3 CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ds.h"

namespace ds {

constexpr int kMaxD = 4;      // d in {2, 3, 4}
constexpr int64_t kDenseMaxPoints = 4096;   // DS_EXPRK3_DENSE: N x N phi-matrices
constexpr int kSlots = 5;     // (s2,l1) (s3,l1) (s3,l2) (sf,l1) (sf,l2)
constexpr int kMaxTerms = 3;

// Split coefficients of one target function phi_l (Section 2 tables).
struct SplitCoeffs {
    int k;                    // number of terms
    int ell_i[kMaxTerms];     // phi index of each term
    double eta[kMaxTerms];
    double alpha[kMaxTerms][kMaxD];
    double eta_im[kMaxTerms];            // imaginary parts (complex scheme; else 0)
    double alpha_im[kMaxTerms][kMaxD];
};
SplitCoeffs split_coeffs(int d, int ell);
SplitCoeffs split_coeffs_cplx(int d, int ell);

// Stage scalar c_s of each slot and target l of each slot.
extern const double kSlotC[kSlots];
extern const int kSlotEll[kSlots];
// Weight multiplying S_s^{(l)} in the step: tau/3, 2tau/3, 4tau/3, tau, 3tau/2 (x tau).
extern const double kSlotW[kSlots];

// Error helpers ----------------------------------------------------------
void set_error(const std::string &msg);
ds_status fail(ds_status st, const std::string &msg);
// The current device is a GB300 (sm_103): DS_OK, else DS_ERR_CUDA (no
// device) or DS_ERR_UNSUPPORTED (another architecture).
ds_status check_device();
#define DS_CUDA_TRY(expr)                                                             \
    do {                                                                              \
        cudaError_t _e = (expr);                                                      \
        if (_e != cudaSuccess)                                                        \
            return ::ds::fail(_e == cudaErrorMemoryAllocation ? DS_ERR_OOM : DS_ERR_CUDA, \
                              std::string(#expr) + ": " + cudaGetErrorString(_e));   \
    } while (0)

// Strided batched FP64 GEMM: C[b] = alpha * A[b] B[b] + beta * C[b] ------
struct DGemm {
    int M, N, K, batch;
    const double *A; int64_t sAm, sAk, sAb;
    const double *B; int64_t sBk, sBn, sBb;
    double *C; int64_t sCm, sCn, sCb;
    double alpha, beta;
};
void launch_dgemm(const DGemm &g, cudaStream_t st);
struct SGemm {
    int M, N, K, batch;
    const float *A; int64_t sAm, sAk, sAb;
    const float *B; int64_t sBk, sBn, sBb;
    float *C; int64_t sCm, sCn, sCb;
    double alpha, beta;
};
void launch_sgemm(const SGemm &g, cudaStream_t st);
void launch_mode_product_f32(int d, const int64_t *n, const float *X, int mu, const float *L,
                             int transpose, float *Y, double alpha, double beta, cudaStream_t st);

// One FP64 mu-mode product Y = X x_mu L (+ beta Y), any mode, as a GEMM.
// L column-major n_mu x n_mu; transpose uses L^T.
void launch_mode_product_f64(int d, const int64_t *n, const double *X, int mu, const double *L,
                             int transpose, double *Y, double alpha, double beta, cudaStream_t st);

// Reaction model ---------------------------------------------------------
struct Model {
    int model;
    double p[8];
};

// Stencil description of K for one component (tridiagonal A_mu only).
struct Stencil {
    int d;
    int64_t n[kMaxD];
    const double *lo[kMaxD], *di[kMaxD], *up[kMaxD];   // device arrays of length n_mu
};

// F = K U + g(U) for both components (FP64, stencil).  Returns #launches.
int launch_rhs_f64(const Stencil *st2, const Model &m, int64_t N, const double *U, double *F,
                   cudaStream_t st);
// D = g(U + w1 a (+ w2 b)) - g(U); b may be null.
void launch_stage_diff_f64(const Model &m, int64_t N, const double *U, const double *a, double w1,
                           const double *b, double w2, double *D, cudaStream_t st);
// U <- (U + w1 a) + w2 b
void launch_final_f64(int64_t N, double *U, const double *a, double w1, const double *b,
                      double w2, cudaStream_t st);
void launch_add_g_f64(const Model &m, int64_t N, const double *U, double *F, cudaStream_t st);
// adjoint helpers (FP64)
void launch_axpy2_f64(int64_t N, const double *U, const double *a, double w1, const double *b, double w2,
                      double *Y, cudaStream_t st);
void launch_gdiff_f64(const Model &m, int64_t N, const double *U, const double *Us, double *D, cudaStream_t st);
void launch_jacT_f64(const Model &m, int64_t N, const double *Us, const double *lam, double *out,
                     cudaStream_t st);
void launch_kronsumT_f64(const Stencil *s2, int64_t N, const double *X, double *Y, cudaStream_t st);
// out[0] += w * sum a.b over n values (block reduction + one atomic per block)
void launch_dot_accum_f64(int64_t n, const double *a, const double *b, double w, double *out,
                          cudaStream_t st);
// out[c] += sum over points of lF_c (F_c - g_c(U)) for c = 0, 1
void launch_dot_kterm_f64(const Model &m, int64_t N, const double *U, const double *F, const double *lF,
                          double *out, cudaStream_t st);
void launch_adjoint_final_f64(const Model &m, int64_t N, const double *U, const double *U2,
                              const double *U3, const double *lam, const double *lU3, const double *lU2,
                              const double *KT, const double *lF, const double *lD2, const double *lD3,
                              double *lam_n, double *dp, cudaStream_t st);

// phi-function evaluation (batched) -------------------------------------
struct PhiJob {
    const double *A;   // device, column-major n x n
    double z;          // scalar multiplying A
    int ell;           // phi index wanted (1 or 2)
    double *out;       // device destination n x n column-major
    double *dout;      // optional: d/ds phi_ell(s zA) at s = 1 = phi_{ell-1} - ell phi_ell
};
ds_status phi_batch_f64(int n, const std::vector<PhiJob> &jobs, cudaStream_t st);

// phi of complex multiples z_b A_b through the real 2n x 2n embedding
// [[Re, -Im], [Im, Re]]; writes the real and imaginary parts.
struct PhiJobC {
    const double *A;   // device, real column-major n x n
    double zr, zi;     // complex scalar multiplying A
    int ell;
    double *out_re, *out_im;
};
ds_status phi_batch_cplx(int n, const std::vector<PhiJobC> &jobs, cudaStream_t st);
// M1 = er Qr - ei Qi, M2 = -(er Qi + ei Qr)  (n x n)
void launch_fold_cplx(int64_t nn, const double *Qr, const double *Qi, double er, double ei, double *M1,
                      double *M2, cudaStream_t st);

// Non-finite scan: sets *flag (device int) to 1 if any entry is NaN/Inf.
void launch_nonfinite_scan(const double *x, int64_t count, int *flag, cudaStream_t st);

// Optional per-launch timing with CUDA events on the launching stream.
// kind: 0 = tensor-core mode product (split BF16), 1 = FP64 mode product,
// 2 = pointwise, 3 = tensor-core mode product with FX operands.
struct Prof {
    struct Rec {
        cudaEvent_t a, b;
        int kind;
        double flops;
        double bytes;   // algorithmic DRAM bytes: compulsory reads of inputs + writes of outputs
    };
    bool on = false;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t take()
    {
        if (pool.empty()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    void begin(cudaStream_t st, int kind, double flops, double bytes = 0.0)
    {
        if (!on) return;
        Rec r{take(), take(), kind, flops, bytes};
        cudaEventRecord(r.a, st);
        recs.push_back(r);
    }
    void end(cudaStream_t st)
    {
        if (!on || recs.empty()) return;
        cudaEventRecord(recs.back().b, st);
    }
    ~Prof()
    {
        for (auto &r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Device-side error word shared by the bounded waits of the tensor-core kernels.
struct DevStatus {
    int timeout;       // set to 1 by a wait that gave up
    int where;         // which wait
    int nonfinite;
    int pad;
};

}  // namespace ds

// Library-owned objects ---------------------------------------------------
struct ds_phi_set {
    int scheme = 0;                         // ds_scheme
    int nslots = 5;                         // 5 (EXPRK3DS_REAL) or 2 (ETD2RKDS)
    int user_d;                             // the caller's grid
    int64_t user_n[ds::kMaxD];
    int d;                                  // the grid of the phi-matrices: the caller's, or for the
    int64_t n[ds::kMaxD];                   // dense scheme one direction of N points (A = K)
    int k;
    double tau;
    ds::SplitCoeffs co[2];                  // [l-1]
    double *A_dev = nullptr;                // copy of A, column-major blocks
    int64_t A_off[2][ds::kMaxD];
    bool tridiag[2];                        // every A_{c,mu} tridiagonal
    double *tri_dev = nullptr;              // [c][mu][3][n_mu]
    int64_t tri_off[2][ds::kMaxD];
    double *P_dev = nullptr;                // FP64 phi-matrices, column-major blocks
    double *dP_dev = nullptr;               // their derivatives w.r.t. a scaling of A (same offsets)
    double *Pim_dev = nullptr;              // complex scheme: imaginary parts (same offsets)
    double *Mf_dev = nullptr;               // complex scheme: last-mode matrices with Re(eta .) folded in
    int64_t Mf_off[2][ds::kSlots][ds::kMaxTerms];
    int64_t P_off[2][ds::kSlots][ds::kMaxTerms][ds::kMaxD];
    int64_t P_count = 0;
};
