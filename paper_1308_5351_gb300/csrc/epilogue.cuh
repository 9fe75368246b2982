// The operator epilogues of a Cauchy sum z = E w (Eqs. (I-B)x, hD-bt, BTx,
// bh, bve and the fused forms of the FBIE listing): from the sums z_r at node
// i, the output entries of the product the job asks for.  Shared by the
// pair-sum reduction and the FMM's L2P.  Internal header.
#pragma once

#include "gnk_internal.h"

namespace gnk {

struct ReduceArgs {
    int N, n, R, chunks, ptype;  // partial type: 0 double2, 1 float2, 2 df32 float4
    double c;
    const double2* p64;
    const float2* p32;
    const float4* pdf;
    const double2* A;
    const double2* q;
    const double* b1;
    const double* d1;
    const double* e;
    double* b1w;  // EPI_EONE_RHS writes diag(B1), diag(D1)
    double* d1w;
    PairJob job;
};

// The epilogue's operands for a job on boundary b; partial sums (chunks of
// type ptype) in b.partial for the pair-sum reduction.
inline ReduceArgs reduce_args(const Boundary& b, const PairJob& job, int chunks, int ptype) {
    ReduceArgs ra;
    ra.N = b.N;
    ra.n = b.n;
    ra.R = job.R;
    ra.chunks = chunks;
    ra.ptype = ptype;
    ra.pdf = static_cast<const float4*>(b.partial);
    ra.c = b.bounded ? 1.0 : -1.0;
    ra.p64 = static_cast<const double2*>(b.partial);
    ra.p32 = static_cast<const float2*>(b.partial);
    ra.A = b.A;
    ra.q = b.q;
    ra.b1 = b.b1;
    ra.d1 = b.d1;
    ra.e = b.e;
    ra.b1w = b.b1;
    ra.d1w = b.d1;
    ra.job = job;
    return ra;
}

// Writes the outputs of epilogue kind `epi` at node i from the sums z0 and
// (a.R = 2) z1.  A caller that knows the kind at compile time passes it as a
// constant, so that only that case is compiled in (a runtime switch over the
// kinds may be evaluated case by case under predication, and every case costs
// FP64 operations on GB300's 2-lane FP64 pipe).
__device__ __forceinline__ void epilogue_apply_as(const ReduceArgs& a, int epi, int i, double2 z0, double2 z1) {
    const PairJob& j = a.job;
    const int N = a.N;
    const double s2n = 2.0 / a.n;
    switch (epi) {
        case EPI_Z:
            j.out_c[i] = z0;
            if (a.R > 1) j.out_c[(size_t)N + i] = z1;
            break;
        case EPI_IMINUSN:
        case EPI_RESID: {
            // f_B(x) = 2x + diag(B1) x - B x, -B x = (2/n) Im(A E(q x))  (Eq. (I-B)x)
            const double2 A = a.A[i];
            const double x = j.ex[i];
            const double fb = 2.0 * x + a.b1[i] * x + s2n * (A.x * z0.y + A.y * z0.x);
            j.out[i] = (epi == EPI_RESID) ? j.rhs[i] - fb : fb;
            break;
        }
        case EPI_M: {
            // f_C(x) = D x - diag(D1) x + Lhat x, D x = -(2/n) Re(A E(q x))  (Eq. hD-bt)
            const double2 A = a.A[i];
            const double x = j.ex[i];
            j.out[i] = -s2n * (A.x * z0.x - A.y * z0.y) - a.d1[i] * x + j.Lx[i];
            break;
        }
        case EPI_ADJ:
        case EPI_RESID_ADJ: {
            // g_B(x) = e x + B^T x + Phat x, B^T x = (2/n) Im(q E(A x))  (Eq. BTx)
            const double2 q = a.q[i];
            const double x = j.ex[i];
            const double gb = a.e[i] * x + s2n * (q.x * z0.y + q.y * z0.x) + j.means[i / a.n];
            j.out[i] = (epi == EPI_RESID_ADJ) ? j.rhs[i] - gb : gb;
            break;
        }
        case EPI_H: {
            // h = (f_C(mu) - f_B(gamma)) / 2  (Eq. bh); z0 = E(q mu), z1 = E(q gamma)
            const double2 A = a.A[i];
            const double mu = j.ex[i];
            const double ga = j.ex2[i];
            const double fc = -s2n * (A.x * z0.x - A.y * z0.y) - a.d1[i] * mu + j.Lx[i];
            const double fb = 2.0 * ga + a.b1[i] * ga + s2n * (A.x * z1.y + A.y * z1.x);
            j.out[i] = 0.5 * (fc - fb);
            break;
        }
        case EPI_EONE_RHS: {
            // z0 = E q (Eone), z1 = E(q gamma): the diagonals, -y and f_B(gamma) at once
            const double2 A = a.A[i];
            const double b1v = -s2n * (A.x * z0.y + A.y * z0.x);
            const double d1v = -s2n * (A.x * z0.x - A.y * z0.y);
            j.out_c[i] = make_double2(z0.x, z0.y);
            a.b1w[i] = b1v;
            a.d1w[i] = d1v;
            const double x = j.ex[i];
            const double fc = -s2n * (A.x * z1.x - A.y * z1.y) - d1v * x + j.Lx[i];
            j.out[i] = -fc;
            j.out2[i] = 2.0 * x + b1v * x + s2n * (A.x * z1.y + A.y * z1.x);
            break;
        }
        case EPI_IMINUSN_T:
        case EPI_RESID_T: {
            // K^T x = 2x + diag(B1) x - B^T x, B^T x = (2/n) Im(q E(A x))  (Eq. BTx)
            const double2 q = a.q[i];
            const double x = j.ex[i];
            const double kt = 2.0 * x + a.b1[i] * x - s2n * (q.x * z0.y + q.y * z0.x);
            j.out[i] = (epi == EPI_RESID_T) ? j.rhs[i] - kt : kt;
            break;
        }
        case EPI_MT: {
            // M^T x = D^T x - diag(D1) x - Lhat x, D^T x = (2/n) Re(q E(A x)), L^T = -L
            const double2 q = a.q[i];
            const double x = j.ex[i];
            j.out[i] = s2n * (q.x * z0.x - q.y * z0.y) - a.d1[i] * x - j.Lx[i];
            break;
        }
        case EPI_RHS_FB: {
            // z = E(q gamma): out = -f_C(gamma) = -y (Eq. y), out2 = f_B(gamma) (kept for h)
            const double2 A = a.A[i];
            const double x = j.ex[i];
            const double fc = -s2n * (A.x * z0.x - A.y * z0.y) - a.d1[i] * x + j.Lx[i];
            j.out[i] = -fc;
            j.out2[i] = 2.0 * x + a.b1[i] * x + s2n * (A.x * z0.y + A.y * z0.x);
            break;
        }
        case EPI_RESID_FC: {
            // out = rhs - f_B(x) and out2 = f_C(x) from the same z = E(q x)
            const double2 A = a.A[i];
            const double x = j.ex[i];
            const double fb = 2.0 * x + a.b1[i] * x + s2n * (A.x * z0.y + A.y * z0.x);
            j.out[i] = j.rhs[i] - fb;
            j.out2[i] = -s2n * (A.x * z0.x - A.y * z0.y) - a.d1[i] * x + j.Lx[i];
            break;
        }
        case EPI_EONE: {
            // diag(B1) = -(2/n) Im(A Eone), diag(D1) = -(2/n) Re(A Eone)  (listing of FBIE);
            // with a second right-hand side z1 = E eta':
            // e = 1 - c - (2/n) Im(E eta') + [(2/n) Im(eta''/eta' - A'/A)]  (Eq. bve),
            // the bracket having been stored in out3 beforehand.
            const double2 A = a.A[i];
            j.out_c[i] = make_double2(z0.x, z0.y);
            j.out[i] = -s2n * (A.x * z0.y + A.y * z0.x);
            j.out2[i] = -s2n * (A.x * z0.x - A.y * z0.y);
            if (a.R > 1) j.out3[i] = 1.0 - a.c - s2n * z1.y + j.out3[i];
            break;
        }
        default:
            break;
    }
}

// The job's own kind, read at run time (the pair-sum reduction).
__device__ __forceinline__ void epilogue_apply(const ReduceArgs& a, int i, double2 z0, double2 z1) {
    epilogue_apply_as(a, a.job.epi, i, z0, z1);
}

}  // namespace gnk
