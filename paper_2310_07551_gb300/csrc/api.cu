// C ABI entry points: validation, object lifetimes, step orchestration and
// CUDA-graph replay.  The arithmetic lives in f64.cu and tc.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "ds_internal.h"
#include "tc.h"

namespace ds {

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
ds_status fail(ds_status st, const std::string &msg)
{
    set_error(msg);
    return st;
}

// ---------------------------------------------------------------------------
// Split coefficients from the closed forms of the paper's tables.
//   d = 2: Table 1, real columns, upper ("+") sign; terms use phi_1, phi_2.
//   d >= 3: Table 3, upper sign in alpha_{1,mu}; terms use phi_1, phi_2,
//          phi_1; eta_{2,d} carries 2^(d-3); alpha is the same in every mu.
// ---------------------------------------------------------------------------
SplitCoeffs split_coeffs(int d, int ell)
{
    SplitCoeffs c{};
    if (d == 2) {
        c.k = 2;
        c.ell_i[0] = 1;
        c.ell_i[1] = 2;
        if (ell == 1) {
            const double r10 = sqrt(10.0);
            c.eta[0] = -1.25;
            c.eta[1] = 9.0;
            c.alpha[0][0] = 4.0 / 3.0 + 4.0 * r10 / 15.0;
            c.alpha[0][1] = 4.0 / 3.0 - 4.0 * r10 / 15.0;
            c.alpha[1][0] = 16.0 / 9.0 + 2.0 * r10 / 9.0;
            c.alpha[1][1] = 16.0 / 9.0 - 2.0 * r10 / 9.0;
        } else {
            const double r33 = sqrt(33.0);
            c.eta[0] = -4.0 / 3.0;
            c.eta[1] = 22.0 / 3.0;
            c.alpha[0][0] = 9.0 / 8.0 + r33 / 8.0;
            c.alpha[0][1] = 9.0 / 8.0 - r33 / 8.0;
            c.alpha[1][0] = 1.5 + 3.0 * r33 / 22.0;
            c.alpha[1][1] = 1.5 - 3.0 * r33 / 22.0;
        }
        return c;
    }
    c.k = 3;
    c.ell_i[0] = 1;
    c.ell_i[1] = 2;
    c.ell_i[2] = 1;
    const double pow2 = ldexp(1.0, d - 3);
    double e_mid, e_off, a_mid, a_off, eta2, alpha2;
    if (ell == 1) {
        const double r = sqrt(2991111.0);
        e_mid = 2243.0 / 1350.0;
        e_off = 440521.0 / 675.0 / r;
        a_mid = 3.0 * 5161.0 / 15869.0;
        a_off = 3.0 * r / 15869.0;
        eta2 = -(12544.0 / 675.0) * pow2;
        alpha2 = 45.0 / 28.0;
    } else {
        const double r = sqrt(2391.0);
        e_mid = 19.0 / 27.0;
        e_off = 151.0 / 27.0 / r;
        a_mid = 3.0 * 121.0 / 490.0;
        a_off = 3.0 * r / 490.0;
        eta2 = -(196.0 / 27.0) * pow2;
        alpha2 = 9.0 / 7.0;
    }
    c.eta[0] = e_mid + e_off;
    c.eta[1] = eta2;
    c.eta[2] = e_mid - e_off;
    for (int mu = 0; mu < d; ++mu) {
        c.alpha[0][mu] = a_mid + a_off;
        c.alpha[1][mu] = alpha2;
        c.alpha[2][mu] = a_mid - a_off;
    }
    return c;
}

// Table 2 (complex two-term split, any d), upper signs; l_1 = 1, l_2 = 2;
// eta_{2,d} carries 2^(d-2); alpha is the same in every direction.
SplitCoeffs split_coeffs_cplx(int d, int ell)
{
    SplitCoeffs c{};
    c.k = 2;
    c.ell_i[0] = 1;
    c.ell_i[1] = 2;
    const double sc = ldexp(1.0, d - 2);
    double e1r, e1i, a1r, a1i, e2r, e2i, a2r, a2i;
    if (ell == 1) {
        const double r2 = sqrt(2.0);
        e1r = 1.75; e1i = 1.5 * r2;
        a1r = 12.0 / 11.0; a1i = -4.0 * r2 / 11.0;
        e2r = -3.0 * sc; e2i = -6.0 * r2 * sc;
        a2r = 4.0 / 3.0; a2i = -2.0 * r2 / 3.0;
    } else {
        const double r3 = sqrt(3.0);
        e1r = 2.0 / 3.0; e1i = 2.0 * r3 / 3.0;
        a1r = 0.75; a1i = -r3 / 4.0;
        e2r = -2.0 / 3.0 * sc; e2i = -8.0 * r3 / 3.0 * sc;
        a2r = 6.0 / 7.0; a2i = -3.0 * r3 / 7.0;
    }
    c.eta[0] = e1r; c.eta_im[0] = e1i;
    c.eta[1] = e2r; c.eta_im[1] = e2i;
    for (int mu = 0; mu < d; ++mu) {
        c.alpha[0][mu] = a1r; c.alpha_im[0][mu] = a1i;
        c.alpha[1][mu] = a2r; c.alpha_im[1][mu] = a2i;
    }
    return c;
}

const double kSlotC[kSlots] = {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 1.0, 1.0};
const int kSlotEll[kSlots] = {1, 1, 2, 1, 2};
const double kSlotW[kSlots] = {1.0 / 3.0, 2.0 / 3.0, 4.0 / 3.0, 1.0, 1.5};

}  // namespace ds

using namespace ds;

// sm_103a (GB300) only: DS_ERR_CUDA without a device, DS_ERR_UNSUPPORTED on another one
ds_status ds::check_device()
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(DS_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3)
        return fail(DS_ERR_UNSUPPORTED, "this library is built for sm_103a (GB300) only");
    return DS_OK;
}

namespace {

int64_t numel(const ds_grid *g)
{
    int64_t N = 1;
    for (int q = 0; q < g->d; ++q) N *= g->n[q];
    return N;
}

ds_status check_grid(const ds_grid *g)
{
    if (!g) return fail(DS_ERR_INVALID_ARG, "grid is NULL");
    if (g->d < 2 || g->d > kMaxD) return fail(DS_ERR_INVALID_ARG, "d must be 2, 3 or 4");
    for (int q = 0; q < g->d; ++q)
        if (g->n[q] < 2 || g->n[q] > (1 << 20))
            return fail(DS_ERR_INVALID_ARG, "n_mu must be in [2, 2^20]");
    if (numel(g) > (int64_t)1 << 34) return fail(DS_ERR_INVALID_ARG, "grid too large");
    return DS_OK;
}


// the precisions with FX operands (scales calibrated per state)
bool is_fx(int prec) { return prec == DS_PREC_F16X10 || prec == DS_PREC_F16X13; }

bool is_tridiagonal(const double *A, int64_t n)
{
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i)
            if ((i > j + 1 || j > i + 1) && A[i + n * j] != 0.0) return false;
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// Plans.
// ---------------------------------------------------------------------------
struct ds_plan {
    ds_grid grid;
    int64_t N;
    int prec;
    Model model;
    const ds_phi_set *set;
    cudaStream_t st = nullptr;            // internal non-blocking stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    double *ws = nullptr;                 // FP64 workspace
    int64_t ws_count = 0;
    float *ws32 = nullptr;                // FP32 path workspace
    float *P32 = nullptr;                 // FP32 copies of the phi-matrices
    DevStatus *status = nullptr;          // device error word
    Stencil sten[2];
    std::map<double *, cudaGraphExec_t> graphs;
    int64_t launches = 0;
    tc::MixedPlan *mixed = nullptr;       // tensor-core path state
    double *bws = nullptr;                // adjoint workspace (24 N doubles), lazily allocated
    Prof prof;                            // optional per-launch event timing
    bool profiling = false;               // ds_step records events when set
    const double *fx_state = nullptr;     // FX plans: the state the scales were last set for
    std::map<double *, cudaGraphExec_t> calib_graphs;   // FX: calibrating first step per state
};

namespace {

// acc (+)= w sum_i eta_i T(X_c, {P[c][slot][i][mu]}) (FP64 path); with
// transpose the matrices are P^T (the adjoint operator S^T).
int tucker_sum_f64x(ds_plan *p, int c, int slot, const double *X, double *acc, double w, bool accumulate,
                    int transpose, double *t1, double *t2, cudaStream_t st)
{
    const ds_phi_set *s = p->set;
    const int d = s->d;
    const SplitCoeffs &co = s->co[s->scheme == DS_ETD2RKDS ? slot : kSlotEll[slot] - 1];
    int launches = 0;
    for (int i = 0; i < co.k; ++i) {
        const double *in = X;
        for (int mu = 0; mu < d; ++mu) {
            const double *L = s->P_dev + s->P_off[c][slot][i][mu];
            const bool last = (mu == d - 1);
            double *out = last ? acc : ((mu % 2 == 0) ? t1 : t2);
            p->prof.begin(st, 1, 2.0 * (double)p->N * (double)s->n[mu]);
            launch_mode_product_f64(d, s->n, in, mu, L, transpose, out, last ? w * co.eta[i] : 1.0,
                                    (last && (i > 0 || accumulate)) ? 1.0 : 0.0, st);
            p->prof.end(st);
            ++launches;
            in = out;
        }
    }
    return launches;
}

// Enqueue sum_i eta_i T(X_c, {P[c][slot][i][mu]}) into acc (FP64 path).
int tucker_sum_f64(ds_plan *p, int c, int slot, const double *X, double *acc, double *t1,
                   double *t2, cudaStream_t st)
{
    return tucker_sum_f64x(p, c, slot, X, acc, 1.0, false, 0, t1, t2, st);
}

// F = K U + g(U) with dense mode products (A not tridiagonal)
int rhs_dense_f64(const ds_plan *p, const double *U, double *F, cudaStream_t st)
{
    const ds_phi_set *s = p->set;
    int launches = 0;
    for (int c = 0; c < 2; ++c)
        for (int mu = 0; mu < s->d; ++mu) {
            launch_mode_product_f64(s->d, s->n, U + c * p->N, mu, s->A_dev + s->A_off[c][mu], 0,
                                    F + c * p->N, 1.0, mu > 0 ? 1.0 : 0.0, st);
            ++launches;
        }
    launch_add_g_f64(p->model, p->N, U, F, st);
    return launches + 1;
}

int enqueue_step_f64(ds_plan *p, double *U, cudaStream_t st)
{
    const int64_t N = p->N;
    const double tau = p->set->tau;
    double *F = p->ws, *a = p->ws + 2 * N, *b = p->ws + 4 * N, *D = p->ws + 6 * N;
    double *t1 = p->ws + 8 * N, *t2 = p->ws + 9 * N;
    int L = 0;
    if (p->set->tridiag[0] && p->set->tridiag[1])
        L += launch_rhs_f64(p->sten, p->model, N, U, F, st);
    else
        L += rhs_dense_f64(p, U, F, st);
    // stage U_{n2}
    for (int c = 0; c < 2; ++c) L += tucker_sum_f64(p, c, 0, F + c * N, a + c * N, t1, t2, st);
    launch_stage_diff_f64(p->model, N, U, a, kSlotW[0] * tau, nullptr, 0.0, D, st);
    ++L;
    // stage U_{n3}
    for (int c = 0; c < 2; ++c) {
        L += tucker_sum_f64(p, c, 1, F + c * N, a + c * N, t1, t2, st);
        L += tucker_sum_f64(p, c, 2, D + c * N, b + c * N, t1, t2, st);
    }
    launch_stage_diff_f64(p->model, N, U, a, kSlotW[1] * tau, b, kSlotW[2] * tau, D, st);
    ++L;
    // final approximation
    for (int c = 0; c < 2; ++c) {
        L += tucker_sum_f64(p, c, 3, F + c * N, a + c * N, t1, t2, st);
        L += tucker_sum_f64(p, c, 4, D + c * N, b + c * N, t1, t2, st);
    }
    launch_final_f64(N, U, a, kSlotW[3] * tau, b, kSlotW[4] * tau, st);
    ++L;
    return L;
}

// FP32 CUDA-core path: same sequence as the FP64 path with FP32 operands
int tucker_sum_f32(ds_plan *p, int c, int slot, const float *X, float *acc, float *t1, float *t2,
                   cudaStream_t st)
{
    const ds_phi_set *s = p->set;
    const int d = s->d;
    const SplitCoeffs &co = s->co[kSlotEll[slot] - 1];
    int launches = 0;
    for (int i = 0; i < co.k; ++i) {
        const float *in = X;
        for (int mu = 0; mu < d; ++mu) {
            const float *L = p->P32 + s->P_off[c][slot][i][mu];
            const bool last = (mu == d - 1);
            float *out = last ? acc : ((mu % 2 == 0) ? t1 : t2);
            p->prof.begin(st, 1, 2.0 * (double)p->N * (double)s->n[mu]);
            launch_mode_product_f32(d, s->n, in, mu, L, 0, out, last ? co.eta[i] : 1.0,
                                    (last && i > 0) ? 1.0 : 0.0, st);
            p->prof.end(st);
            ++launches;
            in = out;
        }
    }
    return launches;
}

int enqueue_step_f32(ds_plan *p, double *U, cudaStream_t st)
{
    const int64_t N = p->N;
    const double tau = p->set->tau;
    float *F = p->ws32, *a = F + 2 * N, *b = F + 4 * N, *D = F + 6 * N, *t1 = F + 8 * N, *t2 = F + 9 * N;
    int L = 0;
    p->prof.begin(st, 2, 0.0);
    tc::launch_rhs_f32(p->sten, p->model, N, U, F, st);
    p->prof.end(st);
    ++L;
    for (int c = 0; c < 2; ++c) L += tucker_sum_f32(p, c, 0, F + c * N, a + c * N, t1, t2, st);
    p->prof.begin(st, 2, 0.0);
    tc::launch_stage_f32(p->model, N, U, a, kSlotW[0] * tau, nullptr, 0.0, D, st);
    p->prof.end(st);
    ++L;
    for (int c = 0; c < 2; ++c) {
        L += tucker_sum_f32(p, c, 1, F + c * N, a + c * N, t1, t2, st);
        L += tucker_sum_f32(p, c, 2, D + c * N, b + c * N, t1, t2, st);
    }
    p->prof.begin(st, 2, 0.0);
    tc::launch_stage_f32(p->model, N, U, a, kSlotW[1] * tau, b, kSlotW[2] * tau, D, st);
    p->prof.end(st);
    ++L;
    for (int c = 0; c < 2; ++c) {
        L += tucker_sum_f32(p, c, 3, F + c * N, a + c * N, t1, t2, st);
        L += tucker_sum_f32(p, c, 4, D + c * N, b + c * N, t1, t2, st);
    }
    p->prof.begin(st, 2, 0.0);
    tc::launch_final_f32(N, U, a, kSlotW[3] * tau, b, kSlotW[4] * tau, st);
    p->prof.end(st);
    ++L;
    return L;
}

// Complex scheme (FP64): acc = Re(sum_i eta_i T(X_c, {P_i{mu}})) for real X,
// with complex P = Pr + i Pi.  Mode 1: two real products; middle modes: four;
// the last mode two, against the matrices with Re(eta .) folded in.
int tucker_sum_cplx(ds_plan *p, int c, int slot, const double *X, double *acc, double *w4,
                    cudaStream_t st)
{
    const ds_phi_set *s = p->set;
    const int d = s->d;
    const int64_t N = p->N;
    double *Yr = w4, *Yi = w4 + N, *Zr = w4 + 2 * N, *Zi = w4 + 3 * N;
    int L = 0;
    auto mp = [&](const double *in, int mu, const double *M, double *out, double alpha, double beta) {
        p->prof.begin(st, 1, 2.0 * (double)N * (double)s->n[mu]);
        launch_mode_product_f64(d, s->n, in, mu, M, 0, out, alpha, beta, st);
        p->prof.end(st);
        ++L;
    };
    for (int i = 0; i < s->k; ++i) {
        const int64_t o0 = s->P_off[c][slot][i][0];
        mp(X, 0, s->P_dev + o0, Yr, 1.0, 0.0);
        mp(X, 0, s->Pim_dev + o0, Yi, 1.0, 0.0);
        for (int mu = 1; mu < d - 1; ++mu) {
            const int64_t o = s->P_off[c][slot][i][mu];
            mp(Yr, mu, s->P_dev + o, Zr, 1.0, 0.0);
            mp(Yi, mu, s->Pim_dev + o, Zr, -1.0, 1.0);
            mp(Yr, mu, s->Pim_dev + o, Zi, 1.0, 0.0);
            mp(Yi, mu, s->P_dev + o, Zi, 1.0, 1.0);
            std::swap(Yr, Zr);
            std::swap(Yi, Zi);
        }
        const double *M = s->Mf_dev + s->Mf_off[c][slot][i];
        const int64_t nn = s->n[d - 1] * s->n[d - 1];
        mp(Yr, d - 1, M, acc, 1.0, i > 0 ? 1.0 : 0.0);
        mp(Yi, d - 1, M + nn, acc, 1.0, 1.0);
    }
    return L;
}

int enqueue_step_cplx_f64(ds_plan *p, double *U, cudaStream_t st)
{
    const int64_t N = p->N;
    const double tau = p->set->tau;
    double *F = p->ws, *a = p->ws + 2 * N, *b = p->ws + 4 * N, *D = p->ws + 6 * N, *w4 = p->ws + 8 * N;
    int L = 0;
    if (p->set->tridiag[0] && p->set->tridiag[1])
        L += launch_rhs_f64(p->sten, p->model, N, U, F, st);
    else
        L += rhs_dense_f64(p, U, F, st);
    for (int c = 0; c < 2; ++c) L += tucker_sum_cplx(p, c, 0, F + c * N, a + c * N, w4, st);
    launch_stage_diff_f64(p->model, N, U, a, kSlotW[0] * tau, nullptr, 0.0, D, st);
    ++L;
    for (int c = 0; c < 2; ++c) {
        L += tucker_sum_cplx(p, c, 1, F + c * N, a + c * N, w4, st);
        L += tucker_sum_cplx(p, c, 2, D + c * N, b + c * N, w4, st);
    }
    launch_stage_diff_f64(p->model, N, U, a, kSlotW[1] * tau, b, kSlotW[2] * tau, D, st);
    ++L;
    for (int c = 0; c < 2; ++c) {
        L += tucker_sum_cplx(p, c, 3, F + c * N, a + c * N, w4, st);
        L += tucker_sum_cplx(p, c, 4, D + c * N, b + c * N, w4, st);
    }
    launch_final_f64(N, U, a, kSlotW[3] * tau, b, kSlotW[4] * tau, st);
    ++L;
    return L;
}

// ETD2RKDS (FP64): U2 = U + tau T(F, phi_1), U <- U2 + tau 2^(d-1) T(g(U2) - G, phi_2)
int enqueue_step_etd2_f64(ds_plan *p, double *U, cudaStream_t st)
{
    const int64_t N = p->N;
    const double tau = p->set->tau;
    double *F = p->ws, *a = p->ws + 2 * N, *b = p->ws + 4 * N, *D = p->ws + 6 * N;
    double *t1 = p->ws + 8 * N, *t2 = p->ws + 9 * N;
    int L = 0;
    if (p->set->tridiag[0] && p->set->tridiag[1])
        L += launch_rhs_f64(p->sten, p->model, N, U, F, st);
    else
        L += rhs_dense_f64(p, U, F, st);
    for (int c = 0; c < 2; ++c) L += tucker_sum_f64(p, c, 0, F + c * N, a + c * N, t1, t2, st);
    launch_stage_diff_f64(p->model, N, U, a, tau, nullptr, 0.0, D, st);
    ++L;
    // tucker_sum applies eta = 2^(d-1) of the phi_2 term
    for (int c = 0; c < 2; ++c) L += tucker_sum_f64(p, c, 1, D + c * N, b + c * N, t1, t2, st);
    launch_final_f64(N, U, a, tau, b, tau, st);
    ++L;
    return L;
}

int enqueue_step(ds_plan *p, double *U, cudaStream_t st, bool profile, bool calibrate = false)
{
    p->prof.on = profile;
    int L;
    if (p->set->scheme == DS_ETD2RKDS)
        L = enqueue_step_etd2_f64(p, U, st);
    else if (p->set->scheme == DS_EXPRK3DS_CPLX)
        L = enqueue_step_cplx_f64(p, U, st);
    else if (p->prec == DS_PREC_F64)
        L = enqueue_step_f64(p, U, st);
    else if (p->prec == DS_PREC_F32)
        L = enqueue_step_f32(p, U, st);
    else
        L = tc::enqueue_step_mixed(p->mixed, p->set, p->model, p->sten, U, st, &p->prof, calibrate);
    p->prof.on = false;
    return L;
}

}  // namespace

extern "C" {

const char *ds_last_error(void) { return g_err.c_str(); }

const char *ds_version(void) { return "ds3 0.1 (sm_103a)"; }

ds_status ds_phi_setup(const ds_grid *grid, const double *A, int a_on_device, double tau,
                       ds_phi_set **out, void *stream)
{
    return ds_phi_setup_ex(grid, A, a_on_device, tau, DS_EXPRK3DS_REAL, out, stream);
}

ds_status ds_phi_setup_ex(const ds_grid *grid, const double *A, int a_on_device, double tau, int scheme,
                          ds_phi_set **out, void *stream)
{
    try {
        if (scheme != DS_EXPRK3DS_REAL && scheme != DS_ETD2RKDS && scheme != DS_EXPRK3DS_CPLX &&
            scheme != DS_EXPRK3_DENSE)
            return fail(DS_ERR_INVALID_ARG, "unknown scheme");
        ds_status r = check_grid(grid);
        if (r != DS_OK) return r;
        if (scheme == DS_EXPRK3_DENSE && numel(grid) > kDenseMaxPoints)
            return fail(DS_ERR_UNSUPPORTED, "the dense scheme is limited to 4096 grid points");
        if (!A || !out) return fail(DS_ERR_INVALID_ARG, "A or out is NULL");
        if (!(tau > 0.0) || !isfinite(tau)) return fail(DS_ERR_INVALID_ARG, "tau must be finite and > 0");
        if ((r = check_device()) != DS_OK) return r;
        cudaStream_t st = (cudaStream_t)stream;
        const ds_grid user = *grid;
        int d = grid->d;
        int64_t Acount = 0;
        for (int c = 0; c < 2; ++c)
            for (int mu = 0; mu < d; ++mu) Acount += grid->n[mu] * grid->n[mu];
        std::vector<double> hA(Acount);
        if (a_on_device) {
            DS_CUDA_TRY(cudaMemcpyAsync(hA.data(), A, sizeof(double) * Acount, cudaMemcpyDeviceToHost, st));
            DS_CUDA_TRY(cudaStreamSynchronize(st));
        } else {
            memcpy(hA.data(), A, sizeof(double) * Acount);
        }
        for (int64_t e = 0; e < Acount; ++e)
            if (!isfinite(hA[e])) return fail(DS_ERR_NONFINITE, "A has a non-finite entry");
        // The unsplit scheme is the split machinery on a one-direction problem:
        // A = K_c, the assembled Kronecker sum, one term with eta = alpha = 1.
        ds_grid gin = *grid;
        if (scheme == DS_EXPRK3_DENSE) {
            const int64_t N = numel(grid);
            std::vector<double> hK((size_t)(2 * N * N), 0.0);
            int64_t aoff = 0;
            for (int c = 0; c < 2; ++c) {
                double *K = hK.data() + c * N * N;
                int64_t stride = 1;
                for (int mu = 0; mu < d; ++mu) {
                    const int64_t nm = grid->n[mu];
                    const double *Am = hA.data() + aoff;
                    for (int64_t j = 0; j < N; ++j) {
                        const int64_t jm = (j / stride) % nm;
                        for (int64_t im = 0; im < nm; ++im)
                            K[(j + (im - jm) * stride) + N * j] += Am[im + nm * jm];
                    }
                    stride *= nm;
                    aoff += nm * nm;
                }
            }
            hA.swap(hK);
            Acount = 2 * N * N;
            gin.d = 1;
            gin.n[0] = N;
            for (int q = 1; q < 4; ++q) gin.n[q] = 1;
        }
        grid = &gin;

        ds_phi_set *s = new (std::nothrow) ds_phi_set();
        if (!s) return fail(DS_ERR_OOM, "host allocation");
        s->user_d = d;
        for (int q = 0; q < kMaxD; ++q) s->user_n[q] = q < user.d ? user.n[q] : 1;
        d = grid->d;
        s->d = d;
        for (int q = 0; q < kMaxD; ++q) s->n[q] = q < d ? grid->n[q] : 1;
        s->tau = tau;
        s->scheme = scheme;
        if (scheme == DS_EXPRK3DS_REAL) {
            s->co[0] = split_coeffs(d, 1);
            s->co[1] = split_coeffs(d, 2);
            s->nslots = kSlots;
        } else if (scheme == DS_EXPRK3DS_CPLX) {
            s->co[0] = split_coeffs_cplx(d, 1);
            s->co[1] = split_coeffs_cplx(d, 2);
            s->nslots = kSlots;
        } else if (scheme == DS_EXPRK3_DENSE) {
            for (int l = 1; l <= 2; ++l) {
                SplitCoeffs &c = s->co[l - 1];
                c = SplitCoeffs{};
                c.k = 1;
                c.ell_i[0] = l;
                c.eta[0] = 1.0;
                c.alpha[0][0] = 1.0;
            }
            s->nslots = kSlots;
        } else {
            // second-order split: phi_l(tau K) ~ l!^(d-1) (x)_mu phi_l(tau A_mu)
            for (int l = 1; l <= 2; ++l) {
                SplitCoeffs &c = s->co[l - 1];
                c = SplitCoeffs{};
                c.k = 1;
                c.ell_i[0] = l;
                c.eta[0] = l == 1 ? 1.0 : ldexp(1.0, d - 1);
                for (int mu = 0; mu < d; ++mu) c.alpha[0][mu] = 1.0;
            }
            s->nslots = 2;
        }
        s->k = s->co[0].k;
        // A copy + tridiagonal bands
        int64_t off = 0, toff = 0;
        for (int c = 0; c < 2; ++c) {
            s->tridiag[c] = true;
            for (int mu = 0; mu < d; ++mu) {
                s->A_off[c][mu] = off;
                s->tri_off[c][mu] = toff;
                if (!is_tridiagonal(hA.data() + off, grid->n[mu])) s->tridiag[c] = false;
                off += grid->n[mu] * grid->n[mu];
                toff += 3 * grid->n[mu];
            }
        }
        std::vector<double> htri(toff, 0.0);
        for (int c = 0; c < 2; ++c)
            for (int mu = 0; mu < d; ++mu) {
                const int64_t n = grid->n[mu];
                const double *Am = hA.data() + s->A_off[c][mu];
                double *lo = htri.data() + s->tri_off[c][mu], *di = lo + n, *up = lo + 2 * n;
                for (int64_t i = 0; i < n; ++i) {
                    lo[i] = i > 0 ? Am[i + n * (i - 1)] : 0.0;
                    di[i] = Am[i + n * i];
                    up[i] = i + 1 < n ? Am[i + n * (i + 1)] : 0.0;
                }
            }
        // phi-matrix layout [c][slot][i][mu]
        int64_t poff = 0;
        for (int c = 0; c < 2; ++c)
            for (int q = 0; q < s->nslots; ++q)
                for (int i = 0; i < s->k; ++i)
                    for (int mu = 0; mu < d; ++mu) {
                        s->P_off[c][q][i][mu] = poff;
                        poff += grid->n[mu] * grid->n[mu];
                    }
        s->P_count = poff;
        cudaError_t e1 = cudaMalloc(&s->A_dev, sizeof(double) * Acount);
        cudaError_t e2 = cudaMalloc(&s->tri_dev, sizeof(double) * toff);
        cudaError_t e3 = cudaMalloc(&s->P_dev, sizeof(double) * poff);
        // derivatives feed the adjoint's diffusion-scaling gradient (EXPRK3DS_REAL only)
        cudaError_t e4 = scheme == DS_EXPRK3DS_REAL ? cudaMalloc(&s->dP_dev, sizeof(double) * poff) : cudaSuccess;
        cudaError_t e5 = cudaSuccess, e6 = cudaSuccess;
        if (scheme == DS_EXPRK3DS_CPLX) {
            e5 = cudaMalloc(&s->Pim_dev, sizeof(double) * poff);
            int64_t moff = 0;
            for (int c = 0; c < 2; ++c)
                for (int q = 0; q < kSlots; ++q)
                    for (int i = 0; i < s->k; ++i) {
                        s->Mf_off[c][q][i] = moff;
                        moff += 2 * grid->n[d - 1] * grid->n[d - 1];
                    }
            e6 = cudaMalloc(&s->Mf_dev, sizeof(double) * moff);
        }
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess ||
            e5 != cudaSuccess || e6 != cudaSuccess) {
            cudaGetLastError();
            ds_phi_set_destroy(s);
            return fail(DS_ERR_OOM, "phi-set device allocation");
        }
        cudaMemcpyAsync(s->A_dev, hA.data(), sizeof(double) * Acount, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(s->tri_dev, htri.data(), sizeof(double) * toff, cudaMemcpyHostToDevice, st);
        // group the phi jobs by size
        std::map<int64_t, std::vector<PhiJob>> groups;
        for (int c = 0; c < 2; ++c)
            for (int q = 0; q < s->nslots; ++q) {
                // ETD2RKDS: slot 0 = phi_1(tau A), slot 1 = phi_2(tau A)
                const SplitCoeffs &co = s->co[scheme == DS_ETD2RKDS ? q : kSlotEll[q] - 1];
                const double cq = scheme == DS_ETD2RKDS ? 1.0 : kSlotC[q];
                for (int i = 0; i < s->k; ++i)
                    for (int mu = 0; mu < d; ++mu) {
                        PhiJob j;
                        j.A = s->A_dev + s->A_off[c][mu];
                        j.z = cq * tau * co.alpha[i][mu];
                        j.ell = co.ell_i[i];
                        j.out = s->P_dev + s->P_off[c][q][i][mu];
                        j.dout = s->dP_dev ? s->dP_dev + s->P_off[c][q][i][mu] : nullptr;
                        groups[grid->n[mu]].push_back(j);
                    }
            }
        if (scheme == DS_EXPRK3DS_CPLX) {
            std::map<int64_t, std::vector<PhiJobC>> cgroups;
            for (int c = 0; c < 2; ++c)
                for (int q = 0; q < kSlots; ++q) {
                    const SplitCoeffs &co = s->co[kSlotEll[q] - 1];
                    for (int i = 0; i < s->k; ++i)
                        for (int mu = 0; mu < d; ++mu) {
                            PhiJobC j;
                            j.A = s->A_dev + s->A_off[c][mu];
                            j.zr = kSlotC[q] * tau * co.alpha[i][mu];
                            j.zi = kSlotC[q] * tau * co.alpha_im[i][mu];
                            j.ell = co.ell_i[i];
                            j.out_re = s->P_dev + s->P_off[c][q][i][mu];
                            j.out_im = s->Pim_dev + s->P_off[c][q][i][mu];
                            cgroups[grid->n[mu]].push_back(j);
                        }
                }
            for (auto &kv : cgroups) {
                r = phi_batch_cplx((int)kv.first, kv.second, st);
                if (r != DS_OK) { ds_phi_set_destroy(s); return r; }
            }
            // last mode: Re(eta (Yr + i Yi) x_d (Qr + i Qi)) = Yr x_d M1 + Yi x_d M2
            const int64_t nd = grid->n[d - 1], nn = nd * nd;
            for (int c = 0; c < 2; ++c)
                for (int q = 0; q < kSlots; ++q) {
                    const SplitCoeffs &co = s->co[kSlotEll[q] - 1];
                    for (int i = 0; i < s->k; ++i) {
                        const int64_t o = s->P_off[c][q][i][d - 1];
                        double *M = s->Mf_dev + s->Mf_off[c][q][i];
                        launch_fold_cplx(nn, s->P_dev + o, s->Pim_dev + o, co.eta[i], co.eta_im[i], M, M + nn, st);
                    }
                }
            DS_CUDA_TRY(cudaStreamSynchronize(st));
        } else {
            for (auto &kv : groups) {
                r = phi_batch_f64((int)kv.first, kv.second, st);
                if (r != DS_OK) { ds_phi_set_destroy(s); return r; }
            }
        }
        *out = s;
        return DS_OK;
    } catch (const std::exception &ex) {
        return fail(DS_ERR_CUDA, std::string("exception: ") + ex.what());
    }
}

ds_status ds_phi_set_destroy(ds_phi_set *s)
{
    if (!s) return DS_OK;
    cudaFree(s->A_dev);
    cudaFree(s->tri_dev);
    cudaFree(s->P_dev);
    cudaFree(s->dP_dev);
    cudaFree(s->Pim_dev);
    cudaFree(s->Mf_dev);
    delete s;
    return DS_OK;
}

ds_status ds_phi_get(const ds_phi_set *s, int c, int slot, int term, int mu, double *host_out)
{
    if (!s || !host_out) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (c < 0 || c > 1 || slot < 0 || slot >= s->nslots || term < 0 || term >= s->k || mu < 0 || mu >= s->d)
        return fail(DS_ERR_INVALID_ARG, "index out of range");
    const int64_t n = s->n[mu];
    DS_CUDA_TRY(cudaMemcpy(host_out, s->P_dev + s->P_off[c][slot][term][mu], sizeof(double) * n * n,
                           cudaMemcpyDeviceToHost));
    return DS_OK;
}

ds_status ds_phi_get_ex(const ds_phi_set *s, int c, int slot, int term, int mu, int part, double *host_out)
{
    if (!s || !host_out) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (c < 0 || c > 1 || slot < 0 || slot >= s->nslots || term < 0 || term >= s->k || mu < 0 || mu >= s->d)
        return fail(DS_ERR_INVALID_ARG, "index out of range");
    const double *base = part == 0 ? s->P_dev : part == 1 ? s->Pim_dev : part == 2 ? s->dP_dev : nullptr;
    if (!base) return fail(DS_ERR_INVALID_ARG, "this phi-set has no such part");
    const int64_t n = s->n[mu];
    DS_CUDA_TRY(cudaMemcpy(host_out, base + s->P_off[c][slot][term][mu], sizeof(double) * n * n,
                           cudaMemcpyDeviceToHost));
    return DS_OK;
}

ds_status ds_tucker(const ds_grid *grid, const double *X, double *Y, const double *const *L,
                    int transpose, int precision, void *stream)
{
    ds_status r = check_grid(grid);
    if (r != DS_OK) return r;
    if (!X || !Y || !L) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    for (int mu = 0; mu < grid->d; ++mu)
        if (!L[mu]) return fail(DS_ERR_INVALID_ARG, "L[mu] is NULL");
    if ((r = check_device()) != DS_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t N = numel(grid);
    const int d = grid->d;
    if (precision == DS_PREC_BF16X6 || precision == DS_PREC_BF16X6C)
        return tc::tucker_mixed(grid, X, Y, L, transpose, st, precision == DS_PREC_BF16X6C);
    if (precision == DS_PREC_F16X10 || precision == DS_PREC_F16X13) return tc::tucker_fx(grid, X, Y, L, transpose, st);
    if (precision == DS_PREC_F32) {
        int64_t pm = 0;
        for (int mu = 0; mu < d; ++mu) pm += grid->n[mu] * grid->n[mu];
        float *w = nullptr;
        DS_CUDA_TRY(cudaMallocAsync(&w, sizeof(float) * (3 * N + pm), st));
        float *x32 = w, *b0 = w + N, *b1 = w + 2 * N, *l32 = w + 3 * N;
        tc::launch_convert_f64_f32(N, X, x32, st);
        const float *in = x32;
        float *pl = l32;
        for (int mu = 0; mu < d; ++mu) {
            tc::launch_convert_f64_f32(grid->n[mu] * grid->n[mu], L[mu], pl, st);
            float *out = (mu % 2 == 0) ? b0 : b1;
            launch_mode_product_f32(d, grid->n, in, mu, pl, transpose, out, 1.0, 0.0, st);
            in = out;
            pl += grid->n[mu] * grid->n[mu];
        }
        tc::launch_convert_f32_f64(N, in, Y, st);
        cudaFreeAsync(w, st);
        DS_CUDA_TRY(cudaGetLastError());
        return DS_OK;
    }
    if (precision != DS_PREC_F64) return fail(DS_ERR_UNSUPPORTED, "unknown precision");
    double *tmp = nullptr;
    DS_CUDA_TRY(cudaMallocAsync(&tmp, sizeof(double) * N * 2, st));
    const double *in = X;
    for (int mu = 0; mu < d; ++mu) {
        double *out = (mu == d - 1) ? Y : tmp + (mu % 2) * N;
        launch_mode_product_f64(d, grid->n, in, mu, L[mu], transpose, out, 1.0, 0.0, st);
        in = out;
    }
    cudaFreeAsync(tmp, st);
    DS_CUDA_TRY(cudaGetLastError());
    return DS_OK;
}

ds_status ds_kronsum(const ds_phi_set *s, int c, const double *X, double *Y, void *stream)
{
    if (!s || !X || !Y || c < 0 || c > 1) return fail(DS_ERR_INVALID_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    for (int mu = 0; mu < s->d; ++mu)
        launch_mode_product_f64(s->d, s->n, X, mu, s->A_dev + s->A_off[c][mu], 0, Y, 1.0,
                                mu > 0 ? 1.0 : 0.0, st);
    DS_CUDA_TRY(cudaGetLastError());
    return DS_OK;
}

ds_status ds_plan_create(const ds_grid *grid, const ds_params *params, const ds_phi_set *set,
                         int precision, ds_plan **out)
{
    try {
        ds_status r = check_grid(grid);
        if (r != DS_OK) return r;
        if (!params || !set || !out) return fail(DS_ERR_INVALID_ARG, "NULL argument");
        if (grid->d != set->user_d) return fail(DS_ERR_INVALID_ARG, "grid does not match the phi-set");
        for (int q = 0; q < grid->d; ++q)
            if (grid->n[q] != set->user_n[q]) return fail(DS_ERR_INVALID_ARG, "grid does not match the phi-set");
        if (params->model < 0 || params->model > 2) return fail(DS_ERR_INVALID_ARG, "unknown model");
        for (int q = 0; q < 8; ++q)
            if (!isfinite(params->p[q])) return fail(DS_ERR_INVALID_ARG, "non-finite model parameter");
        if (precision != DS_PREC_F64 && precision != DS_PREC_BF16X6 && precision != DS_PREC_F32 &&
            precision != DS_PREC_BF16X6C && precision != DS_PREC_F16X10 && precision != DS_PREC_F16X13)
            return fail(DS_ERR_UNSUPPORTED, "unknown precision");
        if (set->scheme != DS_EXPRK3DS_REAL && precision != DS_PREC_F64)
            return fail(DS_ERR_UNSUPPORTED, "ETD2RKDS, EXPRK3DS_CPLX and dense EXPRK3 plans are FP64 only");
        if ((r = check_device()) != DS_OK) return r;
        ds_plan *p = new (std::nothrow) ds_plan();
        if (!p) return fail(DS_ERR_OOM, "host allocation");
        p->grid = *grid;
        p->N = numel(grid);
        p->prec = precision;
        p->model.model = params->model;
        for (int q = 0; q < 8; ++q) p->model.p[q] = params->p[q];
        p->set = set;
        for (int c = 0; c < 2; ++c) {
            p->sten[c].d = set->d;
            for (int mu = 0; mu < kMaxD; ++mu) {
                p->sten[c].n[mu] = mu < set->d ? set->n[mu] : 1;
                const double *base = set->tri_dev + (mu < set->d ? set->tri_off[c][mu] : 0);
                p->sten[c].lo[mu] = base;
                p->sten[c].di[mu] = base + p->sten[c].n[mu];
                p->sten[c].up[mu] = base + 2 * p->sten[c].n[mu];
            }
        }
        auto cleanup = [&](ds_status st, const char *m) { ds_plan_destroy(p); return fail(st, m); };
        if (cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess)
            return cleanup(DS_ERR_CUDA, "stream/event creation");
        if (cudaMalloc(&p->status, sizeof(DevStatus)) != cudaSuccess)
            return cleanup(DS_ERR_OOM, "status word");
        cudaMemset(p->status, 0, sizeof(DevStatus));
        if (precision == DS_PREC_F64) {
            p->ws_count = (set->scheme == DS_EXPRK3DS_CPLX ? 12 : 10) * p->N;
            if (cudaMalloc(&p->ws, sizeof(double) * p->ws_count) != cudaSuccess) {
                cudaGetLastError();
                return cleanup(DS_ERR_OOM, "FP64 workspace");
            }
        } else if (precision == DS_PREC_F32) {
            if (!set->tridiag[0] || !set->tridiag[1])
                return cleanup(DS_ERR_UNSUPPORTED, "reduced-precision paths need tridiagonal A_mu (use DS_PREC_F64)");
            if (cudaMalloc(&p->ws32, sizeof(float) * 10 * p->N) != cudaSuccess ||
                cudaMalloc(&p->P32, sizeof(float) * set->P_count) != cudaSuccess) {
                cudaGetLastError();
                return cleanup(DS_ERR_OOM, "FP32 workspace");
            }
            tc::launch_convert_f64_f32(set->P_count, set->P_dev, p->P32, 0);
        } else {
            r = tc::mixed_plan_create(grid, set, p->status, &p->mixed, precision == DS_PREC_BF16X6C,
                                      precision == DS_PREC_F16X10, precision == DS_PREC_F16X13);
            if (r != DS_OK) { ds_plan_destroy(p); return r; }
        }
        cudaDeviceSynchronize();
        *out = p;
        return DS_OK;
    } catch (const std::exception &ex) {
        return fail(DS_ERR_CUDA, std::string("exception: ") + ex.what());
    }
}

ds_status ds_step(ds_plan *p, double *U, void *stream)
{
    if (!p || !U) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    // FX plans measure their tensors' scales on the first step of a state
    const bool calib = is_fx(p->prec) && p->fx_state != U;
    p->launches = enqueue_step(p, U, st, p->profiling, calib);
    if (p->launches < 0) return fail(DS_ERR_CUDA, "step enqueue failed");
    p->fx_state = U;
    DS_CUDA_TRY(cudaGetLastError());
    return DS_OK;
}

ds_status ds_integrate(ds_plan *p, double *U, int64_t nsteps, void *stream)
{
    if (!p || !U || nsteps < 0) return fail(DS_ERR_INVALID_ARG, "bad argument");
    if (nsteps == 0) return DS_OK;
    cudaStream_t user = (cudaStream_t)stream;
    // one captured step per state pointer (FX plans: also a calibrating one)
    auto capture = [&](bool calib, cudaGraphExec_t *out) -> ds_status {
        cudaGraph_t g;
        DS_CUDA_TRY(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
        int L = enqueue_step(p, U, p->st, false, calib);
        cudaError_t e = cudaStreamEndCapture(p->st, &g);
        if (e != cudaSuccess || L < 0)
            return fail(DS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        if (!calib) p->launches = L;
        e = cudaGraphInstantiate(out, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(DS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        return DS_OK;
    };
    auto it = p->graphs.find(U);
    if (it == p->graphs.end()) {
        cudaGraphExec_t ex;
        ds_status r = capture(false, &ex);
        if (r != DS_OK) return r;
        it = p->graphs.emplace(U, ex).first;
    }
    const bool calib = is_fx(p->prec) && p->fx_state != U;
    cudaGraphExec_t cex = nullptr;
    if (calib) {
        auto ic = p->calib_graphs.find(U);
        if (ic == p->calib_graphs.end()) {
            ds_status r = capture(true, &cex);
            if (r != DS_OK) return r;
            ic = p->calib_graphs.emplace(U, cex).first;
        }
        cex = ic->second;
    }
    DS_CUDA_TRY(cudaEventRecord(p->ev_in, user));
    DS_CUDA_TRY(cudaStreamWaitEvent(p->st, p->ev_in, 0));
    for (int64_t s = 0; s < nsteps; ++s) DS_CUDA_TRY(cudaGraphLaunch(s == 0 && cex ? cex : it->second, p->st));
    p->fx_state = U;
    DS_CUDA_TRY(cudaEventRecord(p->ev_out, p->st));
    DS_CUDA_TRY(cudaStreamWaitEvent(user, p->ev_out, 0));
    return DS_OK;
}

ds_status ds_integrate_ckpt(ds_plan *p, double *U, int64_t nsteps, int64_t ckpt_every, double *ckpt,
                            void *stream)
{
    if (!p || !U || nsteps < 0 || ckpt_every <= 0) return fail(DS_ERR_INVALID_ARG, "bad argument");
    if (nsteps >= ckpt_every && !ckpt) return fail(DS_ERR_INVALID_ARG, "NULL checkpoint buffer");
    const int64_t n2 = 2 * p->N;
    int64_t done = 0, j = 0;
    while (done < nsteps) {
        const int64_t m = std::min(ckpt_every, nsteps - done);
        ds_status r = ds_integrate(p, U, m, stream);
        if (r != DS_OK) return r;
        done += m;
        if (m == ckpt_every) {
            DS_CUDA_TRY(cudaMemcpyAsync(ckpt + j * n2, U, sizeof(double) * n2, cudaMemcpyDeviceToDevice,
                                        (cudaStream_t)stream));
            ++j;
        }
    }
    return DS_OK;
}

// dscale[c] += w sum_i eta_i sum_mu < lam_s_c, T(X_c, P with P_mu -> dP_mu) >
static void dscale_family(ds_plan *p, int c, int slot, const double *X, const double *lam_s, double w,
                          double *out, double *t1, double *t2, double *dscale, cudaStream_t st)
{
    const ds_phi_set *s = p->set;
    const int d = s->d;
    const SplitCoeffs &co = s->co[kSlotEll[slot] - 1];
    for (int i = 0; i < co.k; ++i)
        for (int md = 0; md < d; ++md) {
            const double *in = X;
            for (int mu = 0; mu < d; ++mu) {
                const double *L = (mu == md ? s->dP_dev : s->P_dev) + s->P_off[c][slot][i][mu];
                double *o = (mu == d - 1) ? out : ((mu % 2 == 0) ? t1 : t2);
                launch_mode_product_f64(d, s->n, in, mu, L, 0, o, 1.0, 0.0, st);
                in = o;
            }
            launch_dot_accum_f64(p->N, lam_s, out, w * co.eta[i], dscale + c, st);
        }
}

ds_status ds_step_backward(ds_plan *p, const double *U, const double *lam, double *lam_n, double *dparams,
                           double *dscale, void *stream)
{
    if (!p || !U || !lam || !lam_n) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (lam_n == lam || lam_n == U) return fail(DS_ERR_INVALID_ARG, "lam_n must not alias U or lam");
    if (p->prec != DS_PREC_F64) return fail(DS_ERR_UNSUPPORTED, "the adjoint step needs an FP64 plan");
    if (p->set->scheme != DS_EXPRK3DS_REAL) return fail(DS_ERR_UNSUPPORTED, "the adjoint covers EXPRK3DS_REAL");
    const int64_t N = p->N;
    if (!p->bws) {
        cudaError_t e = cudaMalloc(&p->bws, sizeof(double) * 24 * N);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p->bws = nullptr;
            return fail(DS_ERR_OOM, "adjoint workspace");
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    const double tau = p->set->tau;
    double *F = p->bws, *a = F + 2 * N, *b = F + 4 * N, *D2 = F + 6 * N, *U2 = F + 8 * N, *U3 = F + 10 * N;
    double *lF = F + 12 * N, *lD3 = F + 14 * N, *lD2 = F + 16 * N, *lU3 = F + 18 * N, *lU2 = F + 20 * N;
    double *t1 = F + 22 * N, *t2 = F + 23 * N;
    const Model &m = p->model;
    const bool tri = p->set->tridiag[0] && p->set->tridiag[1];
    // forward recomputation of F, U2, D2, U3
    if (tri)
        launch_rhs_f64(p->sten, m, N, U, F, st);
    else
        rhs_dense_f64(p, U, F, st);
    for (int c = 0; c < 2; ++c) tucker_sum_f64(p, c, 0, F + c * N, a + c * N, t1, t2, st);
    launch_axpy2_f64(N, U, a, kSlotW[0] * tau, nullptr, 0.0, U2, st);
    launch_gdiff_f64(m, N, U, U2, D2, st);
    for (int c = 0; c < 2; ++c) {
        tucker_sum_f64(p, c, 1, F + c * N, a + c * N, t1, t2, st);
        tucker_sum_f64(p, c, 2, D2 + c * N, b + c * N, t1, t2, st);
    }
    launch_axpy2_f64(N, U, a, kSlotW[1] * tau, b, kSlotW[2] * tau, U3, st);
    // reverse sweep
    for (int c = 0; c < 2; ++c) {
        tucker_sum_f64x(p, c, 3, lam + c * N, lF + c * N, kSlotW[3] * tau, false, 1, t1, t2, st);
        tucker_sum_f64x(p, c, 4, lam + c * N, lD3 + c * N, kSlotW[4] * tau, false, 1, t1, t2, st);
    }
    launch_jacT_f64(m, N, U3, lD3, lU3, st);
    for (int c = 0; c < 2; ++c) {
        tucker_sum_f64x(p, c, 1, lU3 + c * N, lF + c * N, kSlotW[1] * tau, true, 1, t1, t2, st);
        tucker_sum_f64x(p, c, 2, lU3 + c * N, lD2 + c * N, kSlotW[2] * tau, false, 1, t1, t2, st);
    }
    launch_jacT_f64(m, N, U2, lD2, lU2, st);
    for (int c = 0; c < 2; ++c)
        tucker_sum_f64x(p, c, 0, lU2 + c * N, lF + c * N, kSlotW[0] * tau, true, 1, t1, t2, st);
    if (dscale) {
        // through K (F = s K U + G) and through every phi-matrix; a and b are
        // free after U3: b <- D3 = g(U3) - g(U), a holds one Tucker output
        launch_dot_kterm_f64(m, N, U, F, lF, dscale, st);
        launch_gdiff_f64(m, N, U, U3, b, st);
        for (int c = 0; c < 2; ++c) {
            const double *Fc = F + c * N;
            double *o = a + c * N;
            dscale_family(p, c, 0, Fc, lU2 + c * N, kSlotW[0] * tau, o, t1, t2, dscale, st);
            dscale_family(p, c, 1, Fc, lU3 + c * N, kSlotW[1] * tau, o, t1, t2, dscale, st);
            dscale_family(p, c, 2, D2 + c * N, lU3 + c * N, kSlotW[2] * tau, o, t1, t2, dscale, st);
            dscale_family(p, c, 3, Fc, lam + c * N, kSlotW[3] * tau, o, t1, t2, dscale, st);
            dscale_family(p, c, 4, b + c * N, lam + c * N, kSlotW[4] * tau, o, t1, t2, dscale, st);
        }
    }
    // K^T lam_F into F's storage
    if (tri) {
        launch_kronsumT_f64(p->sten, N, lF, F, st);
    } else {
        for (int c = 0; c < 2; ++c)
            for (int mu = 0; mu < p->set->d; ++mu)
                launch_mode_product_f64(p->set->d, p->set->n, lF + c * N, mu,
                                        p->set->A_dev + p->set->A_off[c][mu], 1, F + c * N, 1.0,
                                        mu > 0 ? 1.0 : 0.0, st);
    }
    launch_adjoint_final_f64(m, N, U, U2, U3, lam, lU3, lU2, F, lF, lD2, lD3, lam_n, dparams, st);
    DS_CUDA_TRY(cudaGetLastError());
    return DS_OK;
}

ds_status ds_plan_sync(ds_plan *p, const double *U, int check_state)
{
    if (!p) return fail(DS_ERR_INVALID_ARG, "NULL plan");
    DS_CUDA_TRY(cudaStreamSynchronize(p->st));
    DS_CUDA_TRY(cudaDeviceSynchronize());
    if (check_state && U) {
        launch_nonfinite_scan(U, 2 * p->N, &p->status->nonfinite, p->st);
        DS_CUDA_TRY(cudaStreamSynchronize(p->st));
    }
    DevStatus h{};
    DS_CUDA_TRY(cudaMemcpy(&h, p->status, sizeof(h), cudaMemcpyDeviceToHost));
    if (h.timeout)
        return fail(DS_ERR_TIMEOUT, "a tensor-core pipeline wait gave up (site " + std::to_string(h.where) + ")");
    if (h.nonfinite) {
        cudaMemset(&p->status->nonfinite, 0, sizeof(int));
        return fail(DS_ERR_NONFINITE, "state holds NaN/Inf");
    }
    if (p->mixed && tc::mixed_plan_fx_overflow(p->mixed, true) > 0)
        return fail(DS_ERR_NONFINITE,
                    "an FX tensor left the FP16 range of its parts (grew ~32x or more past its scale within one step)");
    return DS_OK;
}

int64_t ds_plan_kernels_per_step(const ds_plan *p) { return p ? p->launches : -1; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent instances: one CUDA graph forks every instance's
// steps onto its own captured stream and joins them, so the kernels of
// different instances run concurrently on the GPU's SMs and one graph launch
// advances the whole batch.
// ---------------------------------------------------------------------------
struct ds_batch {
    int ninst = 0;
    std::vector<ds_phi_set *> sets;
    std::vector<ds_plan *> plans;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr, ev_in = nullptr, ev_out = nullptr;
    struct Graph {
        std::vector<double *> U;
        int steps;
        cudaGraphExec_t exec;
        tc::MixedGroup *group = nullptr;   // grouped launches' tables for these state pointers
    };
    std::vector<Graph> graphs;
    int64_t launches_per_step = 0;
    int force_fused[3] = {-1, -1, -1};   // ds_batch_set_fusion
};

namespace {
ds_status batch_graph(ds_batch *b, double *const *U, int steps, cudaGraphExec_t *out)
{
    for (auto &g : b->graphs) {
        if (g.steps != steps) continue;
        bool same = true;
        for (int i = 0; i < b->ninst && same; ++i) same = (g.U[i] == U[i]);
        if (same) { *out = g.exec; return DS_OK; }
    }
    // split-BF16 batches: per step, every instance's F = K U + g(U) in one
    // grouped launch (else each on its own stream), then each mode product of
    // all instances as one grouped launch;
    // other precisions: each instance's steps on its own stream
    bool grouped = true;
    for (auto *p : b->plans) grouped = grouped && p->mixed != nullptr;
    tc::MixedGroup *G = nullptr;
    if (grouped) {
        std::vector<tc::MixedPlan *> mps;
        std::vector<double *> Us(U, U + b->ninst);
        std::vector<Model> models;
        for (auto *p : b->plans) {
            mps.push_back(p->mixed);
            models.push_back(p->model);
        }
        // the group's creation times launches on the plans' work buffers:
        // nothing of an earlier graph may still be running on them
        cudaStreamSynchronize(b->origin);
        ds_status r = tc::mixed_group_create(mps, Us, models, b->force_fused, &G);
        if (r != DS_OK) return r;
    }
    cudaGraph_t graph;
    DS_CUDA_TRY(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    int64_t L = 0;
    bool bad = false;
    if (grouped) {
        for (int k = 0; k < steps; ++k) {
            L += tc::mixed_group_enqueue_rescale(G, b->origin);   // FX batches
            const int lr = tc::mixed_group_enqueue_rhs(G, b->origin);
            L += lr;
            if (!lr) {
                cudaEventRecord(b->fork, b->origin);
                for (int i = 0; i < b->ninst; ++i) {
                    cudaStream_t s = b->streams[i];
                    cudaStreamWaitEvent(s, b->fork, 0);
                    L += tc::enqueue_rhs_mixed(b->plans[i]->mixed, b->plans[i]->model, U[i], s);
                    cudaEventRecord(b->join[i], s);
                    cudaStreamWaitEvent(b->origin, b->join[i], 0);
                }
            }
            L += tc::mixed_group_enqueue(G, b->origin, nullptr);
        }
    } else {
        cudaEventRecord(b->fork, b->origin);
        for (int i = 0; i < b->ninst; ++i) {
            cudaStream_t s = b->streams[i];
            cudaStreamWaitEvent(s, b->fork, 0);
            for (int k = 0; k < steps; ++k) {
                int l = enqueue_step(b->plans[i], U[i], s, false);
                if (l < 0) bad = true;
                L += l;
            }
            cudaEventRecord(b->join[i], s);
            cudaStreamWaitEvent(b->origin, b->join[i], 0);
        }
    }
    cudaError_t e = cudaStreamEndCapture(b->origin, &graph);
    if (e != cudaSuccess || bad) {
        tc::mixed_group_destroy(G);
        return fail(DS_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t ex;
    e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        tc::mixed_group_destroy(G);
        return fail(DS_ERR_CUDA, std::string("batch instantiate: ") + cudaGetErrorString(e));
    }
    b->launches_per_step = L / steps;
    b->graphs.push_back({std::vector<double *>(U, U + b->ninst), steps, ex, G});
    *out = ex;
    return DS_OK;
}
}  // namespace

extern "C" {

ds_status ds_batch_destroy(ds_batch *b)
{
    if (!b) return DS_OK;
    if (b->origin) cudaStreamSynchronize(b->origin);
    for (auto &g : b->graphs) {
        cudaGraphExecDestroy(g.exec);
        tc::mixed_group_destroy(g.group);
    }
    for (auto p : b->plans) ds_plan_destroy(p);
    for (auto s : b->sets) ds_phi_set_destroy(s);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
    return DS_OK;
}

ds_status ds_batch_fusion(const ds_batch *b, int group, int *fused, float *ms_fused, float *ms_separate)
{
    if (!b || !fused || !ms_fused || !ms_separate) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (group < 0 || group > 2) return fail(DS_ERR_INVALID_ARG, "group out of range");
    // the choice of the latest graph; the times of the latest one that
    // measured them (later graphs of the same batch replay the choice)
    bool any = false;
    *ms_fused = *ms_separate = 0.f;
    for (const auto &g : b->graphs) {
        if (!g.group) continue;
        float a = 0.f, s = 0.f;
        tc::mixed_group_fusion(g.group, group, fused, &a, &s);
        if (a > 0.f) {
            *ms_fused = a;
            *ms_separate = s;
        }
        any = true;
    }
    if (!any) return fail(DS_ERR_UNSUPPORTED, "no grouped launches built (split-BF16 batches, after an integrate)");
    return DS_OK;
}

ds_status ds_batch_tile_order(const ds_batch *b, int group, int *order, float *times_ms)
{
    if (!b || !order || !times_ms) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (group < 0 || group > 2) return fail(DS_ERR_INVALID_ARG, "group out of range");
    bool any = false;
    times_ms[0] = times_ms[1] = 0.f;
    for (const auto &g : b->graphs) {
        if (!g.group) continue;
        float t[2];
        tc::mixed_group_tile_order(g.group, group, order, t);
        if (t[0] > 0.f) {
            times_ms[0] = t[0];
            times_ms[1] = t[1];
        }
        any = true;
    }
    if (!any) return fail(DS_ERR_UNSUPPORTED, "no grouped launches built (split-BF16 batches, after an integrate)");
    return DS_OK;
}

ds_status ds_batch_set_fusion(ds_batch *b, int group, int fused)
{
    if (!b) return fail(DS_ERR_INVALID_ARG, "NULL batch");
    if (group < 0 || group > 2 || fused < -1 || fused > 1) return fail(DS_ERR_INVALID_ARG, "group or choice out of range");
    if (b->origin) cudaStreamSynchronize(b->origin);
    b->force_fused[group] = fused;
    // captured steps hold the previous launch sequence
    for (auto &g : b->graphs) {
        cudaGraphExecDestroy(g.exec);
        tc::mixed_group_destroy(g.group);
    }
    b->graphs.clear();
    return DS_OK;
}

ds_status ds_batch_create(int ninst, const ds_grid *grids, const double *const *A, const double *tau,
                          const ds_params *params, int precision, ds_batch **out)
{
    if (ninst <= 0 || ninst > 4096 || !grids || !A || !tau || !params || !out)
        return fail(DS_ERR_INVALID_ARG, "bad batch arguments");
    ds_batch *b = new (std::nothrow) ds_batch();
    if (!b) return fail(DS_ERR_OOM, "host allocation");
    b->ninst = ninst;
    for (int i = 0; i < ninst; ++i) {
        ds_phi_set *s = nullptr;
        ds_status r = ds_phi_setup(&grids[i], A[i], 0, tau[i], &s, nullptr);
        if (r != DS_OK) {
            std::string m = g_err;
            ds_batch_destroy(b);
            return fail(r, "instance " + std::to_string(i) + ": " + m);
        }
        b->sets.push_back(s);
        ds_plan *p = nullptr;
        r = ds_plan_create(&grids[i], &params[i], s, precision, &p);
        if (r != DS_OK) {
            std::string m = g_err;
            ds_batch_destroy(b);
            return fail(r, "instance " + std::to_string(i) + ": " + m);
        }
        b->plans.push_back(p);
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            ds_batch_destroy(b);
            return fail(DS_ERR_CUDA, "stream/event creation");
        }
        b->streams.push_back(st);
        b->join.push_back(ev);
    }
    if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        ds_batch_destroy(b);
        return fail(DS_ERR_CUDA, "stream/event creation");
    }
    *out = b;
    return DS_OK;
}

ds_status ds_batch_integrate(ds_batch *b, double *const *U, int64_t nsteps, void *stream)
{
    if (!b || !U || nsteps < 0) return fail(DS_ERR_INVALID_ARG, "bad argument");
    for (int i = 0; i < b->ninst; ++i)
        if (!U[i]) return fail(DS_ERR_INVALID_ARG, "U[i] is NULL");
    if (nsteps == 0) return DS_OK;
    cudaStream_t user = (cudaStream_t)stream;
    // FX batches: the first step on a set of states is a calibrating step of
    // each instance (its own launches), which measures every FX tensor before
    // writing it; the grouped graphs then use the previous step's maxima
    bool calib = false;
    for (int i = 0; i < b->ninst; ++i)
        calib = calib || (is_fx(b->plans[i]->prec) && b->plans[i]->fx_state != U[i]);
    if (calib) {
        DS_CUDA_TRY(cudaEventRecord(b->ev_in, user));
        DS_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_in, 0));
        for (int i = 0; i < b->ninst; ++i) {
            if (enqueue_step(b->plans[i], U[i], b->origin, false, true) < 0)
                return fail(DS_ERR_CUDA, "instance " + std::to_string(i) + ": calibrating step");
            b->plans[i]->fx_state = U[i];
        }
        DS_CUDA_TRY(cudaGetLastError());
        DS_CUDA_TRY(cudaEventRecord(b->ev_out, b->origin));
        DS_CUDA_TRY(cudaStreamWaitEvent(user, b->ev_out, 0));
        if (--nsteps == 0) return DS_OK;
    }
    const int chunk = (int)std::min<int64_t>(nsteps, 10);
    cudaGraphExec_t g_chunk = nullptr, g_one = nullptr;
    ds_status r = batch_graph(b, U, chunk, &g_chunk);
    if (r != DS_OK) return r;
    if (nsteps % chunk) {
        r = batch_graph(b, U, 1, &g_one);
        if (r != DS_OK) return r;
    }
    DS_CUDA_TRY(cudaEventRecord(b->ev_in, user));
    DS_CUDA_TRY(cudaStreamWaitEvent(b->origin, b->ev_in, 0));
    for (int64_t k = 0; k < nsteps / chunk; ++k) DS_CUDA_TRY(cudaGraphLaunch(g_chunk, b->origin));
    for (int64_t k = 0; k < nsteps % chunk; ++k) DS_CUDA_TRY(cudaGraphLaunch(g_one, b->origin));
    DS_CUDA_TRY(cudaEventRecord(b->ev_out, b->origin));
    DS_CUDA_TRY(cudaStreamWaitEvent(user, b->ev_out, 0));
    return DS_OK;
}

ds_status ds_batch_sync(ds_batch *b)
{
    if (!b) return fail(DS_ERR_INVALID_ARG, "NULL batch");
    DS_CUDA_TRY(cudaStreamSynchronize(b->origin));
    for (int i = 0; i < b->ninst; ++i) {
        ds_status r = ds_plan_sync(b->plans[i], nullptr, 0);
        if (r != DS_OK) return fail(r, "instance " + std::to_string(i) + ": " + g_err);
    }
    return DS_OK;
}

int64_t ds_batch_kernels_per_step(const ds_batch *b) { return b ? b->launches_per_step : -1; }

ds_status ds_plan_tuning_ex(const ds_plan *p, int group, int mu, int *ksplit, int64_t *tiles, int *tile_n,
                            float *times_ms)
{
    if (!p || !ksplit || !tiles || !tile_n || !times_ms) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (!p->mixed) return fail(DS_ERR_UNSUPPORTED, "only split-BF16 plans are tuned");
    if (tc::mixed_plan_tuning(p->mixed, group, mu, ksplit, tiles, tile_n, times_ms) != 0)
        return fail(DS_ERR_INVALID_ARG, "group or mode out of range");
    return DS_OK;
}

ds_status ds_plan_set_tile_order(ds_plan *p, int group, int mu, int order)
{
    if (!p) return fail(DS_ERR_INVALID_ARG, "NULL plan");
    if (!p->mixed) return fail(DS_ERR_UNSUPPORTED, "only split-BF16 plans have tile orders");
    if (p->st) cudaStreamSynchronize(p->st);
    if (tc::mixed_plan_set_tile_order(p->mixed, group, mu, order) != 0)
        return fail(DS_ERR_INVALID_ARG, "group, mode or order out of range");
    for (auto &kv : p->graphs) cudaGraphExecDestroy(kv.second);
    p->graphs.clear();
    return DS_OK;
}

ds_status ds_plan_tile_order(const ds_plan *p, int group, int mu, int *order, float *times_ms)
{
    if (!p || !order || !times_ms) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (!p->mixed) return fail(DS_ERR_UNSUPPORTED, "only split-BF16 plans are tuned");
    if (tc::mixed_plan_tile_order(p->mixed, group, mu, order, times_ms) != 0)
        return fail(DS_ERR_INVALID_ARG, "group or mode out of range");
    return DS_OK;
}

ds_status ds_plan_streamk_times(const ds_plan *p, int group, int mu, float *times_ms)
{
    if (!p || !times_ms) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (!p->mixed) return fail(DS_ERR_UNSUPPORTED, "only split-BF16 plans are tuned");
    if (tc::mixed_plan_streamk_times(p->mixed, group, mu, times_ms) != 0)
        return fail(DS_ERR_INVALID_ARG, "group or mode out of range");
    return DS_OK;
}

ds_status ds_plan_tuning(const ds_plan *p, int group, int mu, int *ksplit, int64_t *tiles, float *times_ms)
{
    if (!times_ms) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    int tile_n = 0;
    float t16[16];
    ds_status r = ds_plan_tuning_ex(p, group, mu, ksplit, tiles, &tile_n, t16);
    if (r != DS_OK) return r;
    const int w = tile_n == 128 ? 1 : 0;
    for (int k = 0; k < 8; ++k) times_ms[k] = t16[w * 8 + k];
    return DS_OK;
}

ds_status ds_plan_fusion(const ds_plan *p, int group, int *fused, float *ms_fused, float *ms_separate)
{
    if (!p || !fused || !ms_fused || !ms_separate) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (!p->mixed) return fail(DS_ERR_UNSUPPORTED, "only split-BF16 plans fuse epilogues");
    if (tc::mixed_plan_fusion(p->mixed, group, fused, ms_fused, ms_separate) != 0)
        return fail(DS_ERR_INVALID_ARG, "group out of range");
    return DS_OK;
}

ds_status ds_plan_set_fusion(ds_plan *p, int group, int fused)
{
    if (!p) return fail(DS_ERR_INVALID_ARG, "NULL plan");
    if (!p->mixed) return fail(DS_ERR_UNSUPPORTED, "only split-BF16 plans fuse epilogues");
    if (p->st) cudaStreamSynchronize(p->st);
    const int rc = tc::mixed_plan_set_fusion(p->mixed, group, fused);
    if (rc == -2) return fail(DS_ERR_UNSUPPORTED, "DS_PREC_F16X13 plans run the separate stage kernels only");
    if (rc != 0) return fail(DS_ERR_INVALID_ARG, "group out of range");
    // captured steps hold the previous launch sequence
    for (auto &kv : p->graphs) cudaGraphExecDestroy(kv.second);
    p->graphs.clear();
    return DS_OK;
}

ds_status ds_plan_set_tiles(ds_plan *p, int group, int mu, int tile_n, int ksplit)
{
    if (!p) return fail(DS_ERR_INVALID_ARG, "NULL plan");
    if (!p->mixed) return fail(DS_ERR_UNSUPPORTED, "only split-BF16 plans have tile choices");
    if (p->st) cudaStreamSynchronize(p->st);
    const int r = tc::mixed_plan_set_tiles(p->mixed, group, mu, tile_n, ksplit);
    if (r == -1) return fail(DS_ERR_INVALID_ARG, "group, mode or tile width out of range");
    if (r == -2) return fail(DS_ERR_INVALID_ARG, "split factor outside the tuned range (or no stream-K form)");
    for (auto &kv : p->graphs) cudaGraphExecDestroy(kv.second);
    p->graphs.clear();
    return DS_OK;
}

ds_status ds_plan_profile(ds_plan *p, int enable)
{
    if (!p) return fail(DS_ERR_INVALID_ARG, "NULL plan");
    p->profiling = enable != 0;
    return DS_OK;
}

ds_status ds_plan_profile_kinds(ds_plan *p, int nkinds, double *ms, int64_t *launches, double *flops,
                                double *bytes)
{
    if (!p || !ms || !launches || !flops) return fail(DS_ERR_INVALID_ARG, "NULL argument");
    if (nkinds < 1 || nkinds > 4) return fail(DS_ERR_INVALID_ARG, "nkinds must be 1..4");
    for (int k = 0; k < nkinds; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
        flops[k] = 0.0;
        if (bytes) bytes[k] = 0.0;
    }
    for (auto &r : p->prof.recs) {
        DS_CUDA_TRY(cudaEventSynchronize(r.b));
        float t = 0.f;
        DS_CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
        // kind 3 (FX tensor-core launches) counts as kind 0 in a three-kind read
        const int k = r.kind < nkinds ? r.kind : 0;
        ms[k] += t;
        launches[k] += 1;
        flops[k] += r.flops;
        if (bytes) bytes[k] += r.bytes;
        p->prof.pool.push_back(r.a);
        p->prof.pool.push_back(r.b);
    }
    p->prof.recs.clear();
    return DS_OK;
}

ds_status ds_plan_profile_read_ex(ds_plan *p, double *ms, int64_t *launches, double *flops, double *bytes)
{
    return ds_plan_profile_kinds(p, 3, ms, launches, flops, bytes);
}

ds_status ds_plan_profile_read(ds_plan *p, double *ms, int64_t *launches, double *flops)
{
    return ds_plan_profile_read_ex(p, ms, launches, flops, nullptr);
}

ds_status ds_plan_destroy(ds_plan *p)
{
    if (!p) return DS_OK;
    if (p->st) cudaStreamSynchronize(p->st);
    for (auto &kv : p->graphs) cudaGraphExecDestroy(kv.second);
    for (auto &kv : p->calib_graphs) cudaGraphExecDestroy(kv.second);
    if (p->mixed) tc::mixed_plan_destroy(p->mixed);
    cudaFree(p->ws);
    cudaFree(p->bws);
    cudaFree(p->ws32);
    cudaFree(p->P32);
    cudaFree(p->status);
    if (p->ev_in) cudaEventDestroy(p->ev_in);
    if (p->ev_out) cudaEventDestroy(p->ev_out);
    if (p->st) cudaStreamDestroy(p->st);
    delete p;
    return DS_OK;
}

}  // extern "C"
