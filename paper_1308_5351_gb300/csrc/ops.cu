// The discrete operators of Secs. 3 and 4 as sequences of launches on one
// stream: an optional circulant or mean pass, then one pair-sum job whose
// epilogue forms the operator's output.
#include "gnk_internal.h"

namespace gnk {

// y = (2I + diag(B1) - B) x   (Eqs. sys, (I-B)x, f_B)
int op_IminusN(const Boundary& b, const double* x, double* y, int prec, cudaStream_t st,
               const int* done) {
    PairJob j;
    j.R = 1;
    j.mode = W_SCALED;
    j.x[0] = x;
    j.s = b.q;
    j.epi = EPI_IMINUSN;
    j.out = y;
    j.ex = x;
    j.done = done;
    return run_pairsum(b, j, prec, st);
}

// y = (D - diag(D1) + Lhat) x   (Eqs. y, hD-bt, L-bs)
int op_M(const Boundary& b, const double* x, double* y, int prec, cudaStream_t st) {
    GNK_TRY(run_circulant(b, x, b.r3, st));
    PairJob j;
    j.R = 1;
    j.mode = W_SCALED;
    j.x[0] = x;
    j.s = b.q;
    j.epi = EPI_M;
    j.out = y;
    j.ex = x;
    j.Lx = b.r3;
    return run_pairsum(b, j, prec, st);
}

// y = (diag(e) + B^T + Phat) x   (Eqs. sys*, BTx, g_B)
int op_adjoint(const Boundary& b, const double* x, double* y, int prec, cudaStream_t st,
               const int* done) {
    GNK_TRY(run_component_means(b, x, b.means, st));
    PairJob j;
    j.R = 1;
    j.mode = W_SCALED;
    j.x[0] = x;
    j.s = b.A;
    j.epi = EPI_ADJ;
    j.out = y;
    j.ex = x;
    j.means = b.means;
    j.done = done;
    return run_pairsum(b, j, prec, st);
}

// y = (2I + diag(B1) - B)^T x = 2x + diag(B1) x - (2/n) Im(q E(A x))
int op_IminusN_T(const Boundary& b, const double* x, double* y, int prec, cudaStream_t st,
                 const int* done) {
    PairJob j;
    j.R = 1;
    j.mode = W_SCALED;
    j.x[0] = x;
    j.s = b.A;
    j.epi = EPI_IMINUSN_T;
    j.out = y;
    j.ex = x;
    j.done = done;
    return run_pairsum(b, j, prec, st);
}

// y = (D - diag(D1) + Lhat)^T x = (2/n) Re(q E(A x)) - diag(D1) x - Lhat x
int op_MT(const Boundary& b, const double* x, double* y, int prec, cudaStream_t st) {
    GNK_TRY(run_circulant(b, x, b.r3, st));
    PairJob j;
    j.R = 1;
    j.mode = W_SCALED;
    j.x[0] = x;
    j.s = b.A;
    j.epi = EPI_MT;
    j.out = y;
    j.ex = x;
    j.Lx = b.r3;
    return run_pairsum(b, j, prec, st);
}

// r = rhs - A x for the operator `op` (OpId); with fc_out (OP_K only) also
// f_C(x) from the same Cauchy sum.
int op_resid(const Boundary& b, int op, const double* rhs, const double* x, double* r,
             int prec, cudaStream_t st, double* fc_out) {
    if (op != OP_K) fc_out = nullptr;
    if (fc_out) GNK_TRY(run_circulant(b, x, b.r3, st));
    PairJob j;
    j.R = 1;
    j.mode = W_SCALED;
    j.x[0] = x;
    j.ex = x;
    j.rhs = rhs;
    j.out = r;
    if (op == OP_KT) {
        j.s = b.A;
        j.epi = EPI_RESID_T;
    } else if (op == OP_ADJ) {
        GNK_TRY(run_component_means(b, x, b.means, st));
        j.s = b.A;
        j.epi = EPI_RESID_ADJ;
        j.means = b.means;
    } else {
        j.s = b.q;
        j.epi = fc_out ? EPI_RESID_FC : EPI_RESID;
        j.out2 = fc_out;
        j.Lx = b.r3;
    }
    return run_pairsum(b, j, prec, st);
}

// rhs = -y = -(D - diag(D1) + Lhat) gamma and fb = f_B(gamma) from one Cauchy
// sum E(q gamma) (Eqs. y, sys; f_B(gamma) is the second half of h, Eq. bh).
int op_rhs_fb(const Boundary& b, const double* gam, double* rhs, double* fb, int prec,
              cudaStream_t st) {
    GNK_TRY(run_circulant(b, gam, b.r3, st));
    PairJob j;
    j.R = 1;
    j.mode = W_SCALED;
    j.x[0] = gam;
    j.s = b.q;
    j.epi = EPI_RHS_FB;
    j.out = rhs;
    j.out2 = fb;
    j.ex = gam;
    j.Lx = b.r3;
    return run_pairsum(b, j, prec, st);
}

// h = ([D - diag(D1) + Lhat] mu - [2I + diag(B1) - B] gamma) / 2   (Eq. bh);
// both Cauchy sums E(q mu) and E(q gamma) come from one two-RHS launch.
int op_h(const Boundary& b, const double* mu, const double* gam, double* h, cudaStream_t st) {
    GNK_TRY(run_circulant(b, mu, b.r3, st));
    PairJob j;
    j.R = 2;
    j.mode = W_SCALED;
    j.x[0] = mu;
    j.x[1] = gam;
    j.s = b.q;
    j.epi = EPI_H;
    j.out = h;
    j.ex = mu;
    j.ex2 = gam;
    j.Lx = b.r3;
    return run_pairsum(b, j, GNK_PREC_FP64, st);
}

namespace {
__global__ void negate_kernel(double* x, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) x[i] = -x[i];
}
}  // namespace

int ensure_eone(const Boundary& bc, cudaStream_t st) {
    if (!bc.eone_pending) return GNK_OK;
    Boundary& b = const_cast<Boundary&>(bc);  // handle state; calls on a handle do not overlap
    PairJob j;
    j.R = b.has_adjoint ? 2 : 1;
    j.mode = W_COMPLEX;
    j.w[0] = b.q;
    j.w[1] = b.etp;
    j.epi = EPI_EONE;
    j.out_c = b.Eone;
    j.out = b.b1;
    j.out2 = b.d1;
    j.out3 = b.e;
    GNK_TRY(run_pairsum(b, j, b.eone_prec, st));
    b.eone_pending = 0;
    return GNK_OK;
}

int op_eone_rhs_fb(const Boundary& bc, const double* gam, double* rhs, double* fb, int prec,
                   cudaStream_t st) {
    Boundary& b = const_cast<Boundary&>(bc);
    GNK_TRY(run_circulant(b, gam, b.r3, st));
    PairJob j;
    j.R = 2;
    j.mode = W_SCALED;
    j.x[0] = b.ones;
    j.x[1] = gam;
    j.s = b.q;
    j.epi = EPI_EONE_RHS;
    j.out_c = b.Eone;
    j.out = rhs;
    j.out2 = fb;
    j.ex = gam;
    j.Lx = b.r3;
    GNK_TRY(run_pairsum(b, j, prec, st));
    b.eone_pending = 0;
    return GNK_OK;
}

namespace {
__global__ void half_diff_kernel(const double* a, const double* b, double* out, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = 0.5 * (a[i] - b[i]);
}
}  // namespace

// out = (a - b) / 2: h = (f_C(mu) - f_B(gamma)) / 2 (Eq. bh)
int op_half_diff(const double* a, const double* b, double* out, int N, cudaStream_t st) {
    half_diff_kernel<<<(N + 255) / 256, 256, 0, st>>>(a, b, out, N);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    return GNK_OK;
}

int op_negate(double* x, int N, cudaStream_t st) {
    negate_kernel<<<(N + 255) / 256, 256, 0, st>>>(x, N);
    GNK_TRY_CUDA(cudaGetLastError());
    count_launches(1);
    return GNK_OK;
}

}  // namespace gnk
