// rklt_plan.cpp -- host-side plan construction (FP64) and the library's status plumbing.
//
// A plan holds, for block size N and correlation rho, the rounded KLT matrix T
// of Sec. 2.3 (T = floor(alpha K + 1/2), entries in {0, +1, -1}), the diagonal
// normalisation S of Eq. 1, T^{-1}, and the FP32 tables the kernels take as
// parameters.  K is the Markov-1 KLT of Sec. 2.1 in closed form.
#include <atomic>
#include <cmath>
#include <numeric>
#include <cstring>
#include <new>

#include "rklt_internal.h"

namespace rklt {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_wait_ns{4000000000ull};

rklt_status fail(rklt_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

uint64_t wait_timeout_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

int diag_bound(int N, int r) {
    if (r <= 0) return 0;
    int seen = 0;
    for (int d = 0; d < 2 * N - 1; d++) {
        seen += (d < N) ? d + 1 : 2 * N - 1 - d;
        if (seen >= r) return d + 1;
    }
    return 2 * N - 1;
}

namespace {

const double kPi = 3.141592653589793238462643383279502884;

// Sec. 2.1's omega equation tan(N w) = -(1 - rho^2) sin w / ((1 + rho^2) cos w - 2 rho),
// cleared of the tangent's poles by multiplying with cos(N w) * denominator.
double omega_residual(int N, double rho, double w) {
    double c2 = 1.0 + rho * rho, d2 = 1.0 - rho * rho;
    return std::sin(N * w) * (c2 * std::cos(w) - 2.0 * rho) + d2 * std::sin(w) * std::cos(N * w);
}

// Root in (k pi / N, (k+1) pi / N): the residual changes sign across every such
// interval (it equals (1 - rho^2) sin(k pi/N) (-1)^k at the inner ends and has
// the trivial zeros w = 0, pi at the outer ends), so bracketing is safe after
// nudging the outer ends inwards.
double omega_root(int N, double rho, int k) {
    double lo = k * kPi / N, hi = (k + 1) * kPi / N;
    const double nudge = 1e-9 * kPi / N;
    if (k == 0) lo += nudge;
    if (k == N - 1) hi -= nudge;
    double flo = omega_residual(N, rho, lo);
    for (int it = 0; it < 200 && hi - lo > 4e-16 * hi; it++) {
        double mid = lo + 0.5 * (hi - lo);
        double fm = omega_residual(N, rho, mid);
        if (fm == 0.0) return mid;
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    return lo + 0.5 * (hi - lo);
}

// Closed-form KLT (Sec. 2.1): row i, column j
//   k_ij = sqrt(2 / (N + lambda_i)) sin(omega_i (j - (N - 1)/2) + (i + 1) pi / 2)
// (row index = eigen-index, column index = sample), lambda_i = (1 - rho^2) /
// (1 + rho^2 - 2 rho cos omega_i).
std::vector<double> klt(int N, double rho) {
    std::vector<double> K(size_t(N) * N);
    for (int i = 0; i < N; i++) {
        double w = omega_root(N, rho, i);
        double lam = (1.0 - rho * rho) / (1.0 + rho * rho - 2.0 * rho * std::cos(w));
        double a = std::sqrt(2.0 / (N + lam));
        for (int j = 0; j < N; j++)
            K[size_t(i) * N + j] = a * std::sin(w * (j - 0.5 * (N - 1)) + 0.5 * (i + 1) * kPi);
    }
    return K;
}

// In-place FP64 inverse with row pivoting; false when singular.
bool invert(int N, std::vector<double> a, std::vector<double> &inv) {
    inv.assign(size_t(N) * N, 0.0);
    for (int i = 0; i < N; i++) inv[size_t(i) * N + i] = 1.0;
    for (int c = 0; c < N; c++) {
        int p = c;
        for (int i = c + 1; i < N; i++)
            if (std::fabs(a[size_t(i) * N + c]) > std::fabs(a[size_t(p) * N + c])) p = i;
        if (std::fabs(a[size_t(p) * N + c]) < 1e-9) return false;
        if (p != c)
            for (int j = 0; j < N; j++) {
                std::swap(a[size_t(p) * N + j], a[size_t(c) * N + j]);
                std::swap(inv[size_t(p) * N + j], inv[size_t(c) * N + j]);
            }
        double piv = 1.0 / a[size_t(c) * N + c];
        for (int j = 0; j < N; j++) { a[size_t(c) * N + j] *= piv; inv[size_t(c) * N + j] *= piv; }
        for (int i = 0; i < N; i++) {
            if (i == c) continue;
            double f = a[size_t(i) * N + c];
            if (f == 0.0) continue;
            for (int j = 0; j < N; j++) {
                a[size_t(i) * N + j] -= f * a[size_t(c) * N + j];
                inv[size_t(i) * N + j] -= f * inv[size_t(c) * N + j];
            }
        }
    }
    return true;
}

template <int M>
void fill_kparams(Plan &p) {
    p.k.assign(sizeof(PlanK<M>), 0);
    PlanK<M> &k = *reinterpret_cast<PlanK<M> *>(p.k.data());
    for (int i = 0; i < M; i++)
        for (int j = 0; j < M / 2; j++)
            k.T[i][j] = p.kind == 0 ? float(p.T[size_t(i) * M + j]) : float(p.M[size_t(i) * M + j]);
    for (int l = 0; l < M / 2; l++)
        for (int j = 0; j < M; j++) {
            k.Ti[l][j] = float(p.Tinv[size_t(l) * M + j]);
            k.Tih[l][j] = float(p.Tinv[size_t(l) * M + j] / p.s[j]);
        }
    if constexpr (M <= 8) {
        for (int j = 0; j < M; j++)
            for (int l = 0; l < M / 2; l++) k.Td[j][l] = make_float2(k.T[j][l], k.T[j][l]);
        for (int c = 0; c < M / 2; c++)
            for (int j = 0; j < M; j++) k.Tid[c][j] = make_float2(k.Ti[c][j], k.Ti[c][j]);
        if (p.kind == 0)
            for (int i = 0; i < M; i++)
                for (int h = 0; h < M / 4; h++) {
                    uint32_t v = 0;
                    for (int q = 0; q < 4; q++) v |= uint32_t(uint8_t(int8_t(p.T[size_t(i) * M + 4 * h + q]))) << (8 * q);
                    k.T8[i][h] = v;
                }
    }
    for (int i = 0; i < M; i++)
        for (int j = 0; j < M; j++) k.sij[i][j] = float(p.s[i] * p.s[j]);
    for (int i = 0; i < M; i++) k.s[i] = float(p.s[i]);
    // 0, +1, -1 as binary16: 0x0000, 0x3C00, 0xBC00, duplicated into both lanes
    // (rounded plans only; real plans never reach the binary16 kernels)
    for (int i = 0; i < M; i++)
        for (int j = 0; j < M / 2; j++) {
            const int t = p.T[size_t(i) * M + j];
            const uint32_t h = t == 0 ? 0x0000u : (t > 0 ? 0x3C00u : 0xBC00u);
            k.T2[i][j] = h | (h << 16);
        }
    // Parseval weights (rounded plans with T T^T diagonal, N <= 8)
    if constexpr (M <= 8) {
        if (p.kind == 0 && p.orthogonal) {
            long d[M], m = 1;
            for (int i = 0; i < M; i++) {
                d[i] = 0;
                for (int j = 0; j < M; j++) d[i] += long(p.T[size_t(i) * M + j]) * p.T[size_t(i) * M + j];
                m = std::lcm(m, d[i]);
            }
            for (int i = 0; i < M; i++)
                for (int j = 0; j < M; j++) k.pw[i][j] = int32_t((m / d[i]) * (m / d[j]));
            k.pm2 = int32_t(m * m);   // d_i <= M <= 8: m <= 840, m^2 <= 705600
            k.pinv = float(1.0 / double(m * m));
        }
    }
}

rklt_status fill_tables(Plan &p) {
    switch (p.N) {
        case 4: fill_kparams<4>(p); break;
        case 8: fill_kparams<8>(p); break;
        case 16: fill_kparams<16>(p); break;
        case 32: fill_kparams<32>(p); break;
        default: return fail(RKLT_ERR_ARG, "N must be 4, 8, 16 or 32");
    }
    return RKLT_OK;
}

// A plan for an orthonormal real matrix M (rows = basis vectors, with the row
// parity M[i][N-1-j] = (-1)^i M[i][j] that the kernels' butterflies use): S = I,
// inverse M^T.
rklt_status finish_real(Plan &p) {
    const int N = p.N;
    p.T.assign(size_t(N) * N, 0);
    p.s.assign(N, 1.0);
    p.orthogonal = 1;
    p.Tinv.assign(size_t(N) * N, 0.0);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) p.Tinv[size_t(i) * N + j] = p.M[size_t(j) * N + i];
    return fill_tables(p);
}

// Orthonormal DCT-II: M[i][j] = c_i cos(pi (2j + 1) i / (2N)).
std::vector<double> dct2(int N) {
    std::vector<double> M(size_t(N) * N);
    for (int i = 0; i < N; i++) {
        const double c = std::sqrt((i == 0 ? 1.0 : 2.0) / N);
        for (int j = 0; j < N; j++) M[size_t(i) * N + j] = c * std::cos(kPi * (2 * j + 1) * i / (2.0 * N));
    }
    return M;
}

// Validate an integer matrix and complete the plan: S (Eq. 1), T^{-1}, tables.
rklt_status finish(Plan &p) {
    const int N = p.N;
    for (int i = 0; i < N; i++) {
        long nn = 0;
        for (int j = 0; j < N; j++) {
            int t = p.T[size_t(i) * N + j];
            if (t < -1 || t > 1) return fail(RKLT_ERR_DEGENERATE, "T has an entry outside {0, +1, -1}");
            int mirror = p.T[size_t(i) * N + (N - 1 - j)];
            if (mirror != ((i & 1) ? -t : t))
                return fail(RKLT_ERR_DEGENERATE, "T lacks the KLT row parity T[i][N-1-j] = (-1)^i T[i][j]");
            nn += long(t) * t;
        }
        if (nn == 0) return fail(RKLT_ERR_DEGENERATE, "T has an all-zero row");
    }
    // Eq. 1: S = sqrt(diag(T T^T)^{-1}); when T T^T is diagonal this is also
    // sqrt((T T^T)^{-1}), the orthogonal branch.
    p.s.assign(N, 0.0);
    p.orthogonal = 1;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            long acc = 0;
            for (int m = 0; m < N; m++) acc += long(p.T[size_t(i) * N + m]) * p.T[size_t(j) * N + m];
            if (i == j) p.s[i] = 1.0 / std::sqrt(double(acc));
            else if (acc != 0) p.orthogonal = 0;
        }
    std::vector<double> Td(size_t(N) * N);
    for (size_t q = 0; q < Td.size(); q++) Td[q] = p.T[q];
    if (!invert(N, Td, p.Tinv)) return fail(RKLT_ERR_DEGENERATE, "T is singular");
    return fill_tables(p);
}

bool valid_n(int N) { return N == 4 || N == 8 || N == 16 || N == 32; }

}  // namespace
}  // namespace rklt

using namespace rklt;

extern "C" {

const char *rklt_last_error(void) { return g_last_error.c_str(); }

const char *rklt_status_string(rklt_status s) {
    switch (s) {
        case RKLT_OK: return "RKLT_OK";
        case RKLT_ERR_ARG: return "RKLT_ERR_ARG";
        case RKLT_ERR_SHAPE: return "RKLT_ERR_SHAPE";
        case RKLT_ERR_DEGENERATE: return "RKLT_ERR_DEGENERATE";
        case RKLT_ERR_CUDA: return "RKLT_ERR_CUDA";
        case RKLT_ERR_OOM: return "RKLT_ERR_OOM";
        case RKLT_ERR_BUDGET: return "RKLT_ERR_BUDGET";
        case RKLT_ERR_TIMEOUT: return "RKLT_ERR_TIMEOUT";
        case RKLT_ERR_UNSUPPORTED: return "RKLT_ERR_UNSUPPORTED";
        default: return "RKLT_ERR_UNKNOWN";
    }
}

int rklt_version(void) { return 10000; }

void rklt_set_wait_timeout_us(uint32_t us) {
    g_wait_ns.store(us ? uint64_t(us) * 1000ull : 4000000000ull, std::memory_order_relaxed);
}

rklt_status rklt_make_alpha(int N, double rho, double alpha, rklt_plan **out) {
    if (!out) return fail(RKLT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_n(N)) return fail(RKLT_ERR_ARG, "N must be 4, 8, 16 or 32");
    if (!(rho > 0.0 && rho < 1.0)) return fail(RKLT_ERR_ARG, "rho must lie in (0, 1)");
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(RKLT_ERR_ARG, "alpha must be positive");
    rklt_plan *h = new (std::nothrow) rklt_plan;
    if (!h) return fail(RKLT_ERR_OOM, "host allocation failed");
    Plan &p = h->p;
    p.N = N; p.rho = rho; p.alpha = alpha;
    std::vector<double> K = klt(N, rho);
    p.T.resize(size_t(N) * N);
    for (size_t q = 0; q < K.size(); q++) {
        double x = alpha * K[q];
        double fl = std::floor(x);
        if (std::fabs(x - (fl + 0.5)) < 1e-9) {
            delete h;
            return fail(RKLT_ERR_DEGENERATE, "alpha*K has an entry within 1e-9 of a rounding tie");
        }
        double t = std::floor(x + 0.5);  // Eq. 2: round(x) = floor(x + 1/2)
        if (t < -1.0 || t > 1.0) {
            delete h;
            return fail(RKLT_ERR_DEGENERATE, "round(alpha*K) has an entry outside {0, +1, -1}; lower alpha");
        }
        p.T[q] = int8_t(t);
    }
    rklt_status st = finish(p);
    if (st != RKLT_OK) { delete h; return st; }
    *out = h;
    return RKLT_OK;
}

rklt_status rklt_make(int N, double rho, rklt_plan **out) {
    if (!valid_n(N)) {
        if (out) *out = nullptr;
        return fail(RKLT_ERR_ARG, "N must be 4, 8, 16 or 32");
    }
    return rklt_make_alpha(N, rho, 2.0 * std::sqrt(N / 8.0), out);
}

rklt_status rklt_make_from_matrix(int N, const int8_t *h_T, rklt_plan **out) {
    if (!out) return fail(RKLT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_n(N)) return fail(RKLT_ERR_ARG, "N must be 4, 8, 16 or 32");
    if (!h_T) return fail(RKLT_ERR_ARG, "h_T is NULL");
    rklt_plan *h = new (std::nothrow) rklt_plan;
    if (!h) return fail(RKLT_ERR_OOM, "host allocation failed");
    h->p.N = N;
    h->p.T.assign(h_T, h_T + size_t(N) * N);
    rklt_status st = finish(h->p);
    if (st != RKLT_OK) { delete h; return st; }
    *out = h;
    return RKLT_OK;
}

rklt_status rklt_make_klt(int N, double rho, rklt_plan **out) {
    if (!out) return fail(RKLT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_n(N)) return fail(RKLT_ERR_ARG, "N must be 4, 8, 16 or 32");
    if (!(rho > 0.0 && rho < 1.0)) return fail(RKLT_ERR_ARG, "rho must lie in (0, 1)");
    rklt_plan *h = new (std::nothrow) rklt_plan;
    if (!h) return fail(RKLT_ERR_OOM, "host allocation failed");
    h->p.N = N;
    h->p.rho = rho;
    h->p.kind = 1;
    h->p.M = klt(N, rho);
    rklt_status st = finish_real(h->p);
    if (st != RKLT_OK) { delete h; return st; }
    *out = h;
    return RKLT_OK;
}

rklt_status rklt_make_dct(int N, rklt_plan **out) {
    if (!out) return fail(RKLT_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_n(N)) return fail(RKLT_ERR_ARG, "N must be 4, 8, 16 or 32");
    rklt_plan *h = new (std::nothrow) rklt_plan;
    if (!h) return fail(RKLT_ERR_OOM, "host allocation failed");
    h->p.N = N;
    h->p.kind = 2;
    h->p.M = dct2(N);
    rklt_status st = finish_real(h->p);
    if (st != RKLT_OK) { delete h; return st; }
    *out = h;
    return RKLT_OK;
}

int rklt_plan_kind(const rklt_plan *plan) { return plan ? plan->p.kind : -1; }

// Algorithm 1 (Sec. 3): for rho = step, 2 step, ..., 1 - step, T' = round(alpha K_rho)
// (Eq. 2); every T' that differs from the previous one joins the output set.
rklt_status rklt_design_sweep(int N, double alpha, double step, int max_out, int8_t *h_T, double *h_rho_first,
                              double *h_rho_last, int *count) {
    if (!count) return fail(RKLT_ERR_ARG, "count is NULL");
    *count = 0;
    if (!valid_n(N)) return fail(RKLT_ERR_ARG, "N must be 4, 8, 16 or 32");
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(RKLT_ERR_ARG, "alpha must be positive");
    if (!(step > 0.0 && step < 0.5)) return fail(RKLT_ERR_ARG, "step must lie in (0, 0.5)");
    if (max_out < 0 || (max_out > 0 && !h_T)) return fail(RKLT_ERR_ARG, "h_T is NULL");
    std::vector<int8_t> prev;
    const long steps = std::lround(1.0 / step);
    int n = 0;
    for (long k = 1; k < steps; k++) {
        const double rho = k * step;
        const std::vector<double> K = klt(N, rho);
        std::vector<int8_t> T(K.size());
        for (size_t q = 0; q < K.size(); q++) {
            const double t = std::floor(alpha * K[q] + 0.5);
            if (t < -127.0 || t > 127.0) return fail(RKLT_ERR_DEGENERATE, "round(alpha*K) leaves the int8 range");
            T[q] = int8_t(t);
        }
        if (T != prev) {
            if (n < max_out) {
                std::memcpy(h_T + size_t(n) * N * N, T.data(), T.size());
                if (h_rho_first) h_rho_first[n] = rho;
            }
            n++;
            prev = T;
        }
        if (n <= max_out && h_rho_last) h_rho_last[n - 1] = rho;
    }
    *count = n;
    return n > max_out ? fail(RKLT_ERR_BUDGET, "more distinct matrices than max_out; *count holds the total")
                       : RKLT_OK;
}

// Figures of merit of a plan's analysis matrix M (T-hat, or the exact KLT / DCT)
// for the Markov-1 model with correlation rho (Sec. 3.1): unified coding gain, transform
// efficiency, MSE to the exact KLT and total error energy.
rklt_status rklt_figures(const rklt_plan *plan, double rho, double *cg, double *eta, double *mse, double *eps) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    if (!(rho > 0.0 && rho < 1.0)) return fail(RKLT_ERR_ARG, "rho must lie in (0, 1)");
    const Plan &p = plan->p;
    const int N = p.N;
    std::vector<double> M(size_t(N) * N), Minv;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            M[size_t(i) * N + j] = p.kind == 0 ? p.s[i] * p.T[size_t(i) * N + j] : p.M[size_t(i) * N + j];
    if (!invert(N, M, Minv)) return fail(RKLT_ERR_DEGENERATE, "the analysis matrix is singular");
    std::vector<double> R(size_t(N) * N);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) R[size_t(i) * N + j] = std::pow(rho, std::abs(i - j));
    const std::vector<double> K = klt(N, rho);
    if (cg) {  // 10 log10 prod_k (A_k B_k)^(-1/N), A_k = h_k R h_k^T, B_k = ||row k of M^{-1}||^2
        double acc = 0.0;
        for (int k = 0; k < N; k++) {
            double A = 0.0, B = 0.0;
            for (int i = 0; i < N; i++)
                for (int j = 0; j < N; j++) A += M[size_t(k) * N + i] * M[size_t(k) * N + j] * R[size_t(i) * N + j];
            for (int j = 0; j < N; j++) B += Minv[size_t(k) * N + j] * Minv[size_t(k) * N + j];
            acc += std::log10(A * B);
        }
        *cg = -10.0 * acc / N;
    }
    if (eta) {  // 100 sum |r_ii| / sum |r_ij|, r = M R M^T
        double diag = 0.0, all = 0.0;
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) {
                double r = 0.0;
                for (int a = 0; a < N; a++)
                    for (int b = 0; b < N; b++) r += M[size_t(i) * N + a] * R[size_t(a) * N + b] * M[size_t(j) * N + b];
                all += std::fabs(r);
                if (i == j) diag += std::fabs(r);
            }
        *eta = 100.0 * diag / all;
    }
    if (mse) {  // tr((K - M) R (K - M)^T) / N
        double tr = 0.0;
        for (int i = 0; i < N; i++)
            for (int a = 0; a < N; a++)
                for (int b = 0; b < N; b++)
                    tr += (K[size_t(i) * N + a] - M[size_t(i) * N + a]) * R[size_t(a) * N + b] *
                          (K[size_t(i) * N + b] - M[size_t(i) * N + b]);
        *mse = tr / N;
    }
    if (eps) {  // pi ||K - M||_F^2
        double f = 0.0;
        for (size_t q = 0; q < M.size(); q++) f += (K[q] - M[q]) * (K[q] - M[q]);
        *eps = kPi * f;
    }
    return RKLT_OK;
}

rklt_status rklt_plan_matrix(const rklt_plan *plan, double *h_M) {
    if (!plan || !h_M) return fail(RKLT_ERR_ARG, "plan or h_M is NULL");
    const Plan &p = plan->p;
    const int N = p.N;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            h_M[size_t(i) * N + j] = p.kind == 0 ? p.s[i] * p.T[size_t(i) * N + j] : p.M[size_t(i) * N + j];
    return RKLT_OK;
}

void rklt_destroy(rklt_plan *plan) {
    if (plan) rklt::plan_registry_release(&plan->p);
    delete plan;
}

rklt_status rklt_plan_info(const rklt_plan *plan, int8_t *h_T, double *h_s, int *orthogonal,
                           int *N_out, double *alpha_out, double *rho_out) {
    if (!plan) return fail(RKLT_ERR_ARG, "plan is NULL");
    const Plan &p = plan->p;
    if (h_T) std::memcpy(h_T, p.T.data(), p.T.size());
    if (h_s) std::memcpy(h_s, p.s.data(), p.s.size() * sizeof(double));
    if (orthogonal) *orthogonal = p.orthogonal;
    if (N_out) *N_out = p.N;
    if (alpha_out) *alpha_out = p.alpha;
    if (rho_out) *rho_out = p.rho;
    return RKLT_OK;
}

}  // extern "C"
