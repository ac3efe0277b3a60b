// ffb_eig.cu -- Alg. 2 step 4: eigenpairs of the steerable covariance blocks
// C^(k) (p_k x p_k, symmetric, float64) by a batched parallel cyclic Jacobi
// method, one CTA per block.
//
// Each sweep visits every pair (i, j) once through a round-robin schedule of
// pp - 1 rounds of pp/2 disjoint pairs (pp = p rounded up to even; the padding
// row/column is zero and never mixes).  For a pair, tau = (a_jj - a_ii) /
// (2 a_ij), t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2),
// s = t c annihilate a_ij in J^T A J with J = [[c, s], [-s, c]] on (i, j).
// Disjoint rotations commute, so a round applies all row rotations, then all
// column rotations (to A and to the eigenvector matrix V).  The sweep count is
// bounded; a block that does not reach ||offdiag||_F <= 2.3e-16 pp ||A||_F (a
// few float64 ulps per element, the floor the rotations' rounding leaves)
// latches FFB_ERR_NOT_CONVERGED and still returns its current estimate.
#include "ffb_internal.cuh"

#define EIG_MAXP 512          // larger blocks are rejected (p_k <= 255 for L <= 512)
#define EIG_VSHARED_MAXP 110  // beyond this V lives in a global workspace
#define EIG_ASHARED_MAXP 166  // beyond this A does too (its pp x (pp+1) doubles fill 227 KB)
#define EIG_MAX_SWEEPS 40

__global__ void __launch_bounds__(256)
k_jacobi(const double *__restrict__ Cfin, const int *__restrict__ pk_, const int *__restrict__ off_,
         const int *__restrict__ cov_off, double *__restrict__ evals, double *__restrict__ evecs, int *status,
         double *__restrict__ vwork, int ldmax, int aglobal) {
    extern __shared__ double shd[];
    const int k = blockIdx.x;
    const int p = pk_[k];
    const int pp = p + (p & 1);
    const int ld = (vwork ? ldmax : pp + 1);
    // workspace of block k: V [ldmax][ldmax], then A [ldmax][ldmax] when aglobal
    double *wk = vwork ? vwork + (size_t)k * (aglobal ? 2 : 1) * ldmax * ldmax : nullptr;
    double *A = aglobal ? wk + (size_t)ldmax * ldmax : shd;            // [pp][ld]
    double *V = vwork ? wk : A + pp * ld;                              // [pp][ld]
    double *cs = aglobal ? shd : (vwork ? A + (size_t)ldmax * ldmax : V + pp * ld);   // [pp/2][2]
    double *red = cs + pp;            // [256]
    int *pos = (int *)(red + 256);    // [pp]
    int *pair = pos + pp;             // [pp/2][2]
    const int tid = threadIdx.x, nt = blockDim.x;
    const double *C = Cfin + cov_off[k];
    for (int e = tid; e < pp * pp; e += nt) {
        int i = e / pp, j = e % pp;
        A[i * ld + j] = (i < p && j < p) ? C[i * p + j] : 0.0;
        V[i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
    for (int i = tid; i < pp; i += nt) pos[i] = i;
    __syncthreads();
    // ||A||_F
    double loc = 0.0;
    for (int e = tid; e < pp * pp; e += nt) {
        double v = A[(e / pp) * ld + e % pp];
        loc += v * v;
    }
    red[tid] = loc;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    const double fro2 = red[0];
    __syncthreads();
    // ||offdiag||_F <= (2.3e-16 pp) ||A||_F: a few float64 ulps per element,
    // the level the rotations' rounding leaves behind
    const double tol2 = (2.3e-16 * pp) * (2.3e-16 * pp) * fro2;
    bool converged = (pp <= 1) || fro2 == 0.0;
    for (int sweep = 0; sweep <= EIG_MAX_SWEEPS && !converged; ++sweep) {
        // off-diagonal norm
        loc = 0.0;
        for (int e = tid; e < pp * pp; e += nt) {
            int i = e / pp, j = e % pp;
            if (i != j) {
                double v = A[i * ld + j];
                loc += v * v;
            }
        }
        red[tid] = loc;
        __syncthreads();
        for (int s = nt / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] += red[tid + s];
            __syncthreads();
        }
        const double off2 = red[0];
        __syncthreads();
        if (off2 <= tol2) {
            converged = true;
            break;
        }
        if (sweep == EIG_MAX_SWEEPS) break;   // the state after the last sweep was checked
        for (int round = 0; round < pp - 1; ++round) {
            for (int m = tid; m < pp / 2; m += nt) {
                int i = pos[m], j = pos[pp - 1 - m];
                if (i > j) {
                    int t = i;
                    i = j;
                    j = t;
                }
                pair[2 * m] = i;
                pair[2 * m + 1] = j;
                double aij = A[i * ld + j];
                double c = 1.0, s = 0.0;
                if (aij != 0.0) {
                    double tau = (A[j * ld + j] - A[i * ld + i]) / (2.0 * aij);
                    double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                cs[2 * m] = c;
                cs[2 * m + 1] = s;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < (pp / 2) * pp; e += nt) {
                int m = e / pp, col = e % pp;
                int i = pair[2 * m], j = pair[2 * m + 1];
                double c = cs[2 * m], s = cs[2 * m + 1];
                double x = A[i * ld + col], y = A[j * ld + col];
                A[i * ld + col] = c * x - s * y;
                A[j * ld + col] = s * x + c * y;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = tid; e < (pp / 2) * pp; e += nt) {
                int m = e / pp, row = e % pp;
                int i = pair[2 * m], j = pair[2 * m + 1];
                double c = cs[2 * m], s = cs[2 * m + 1];
                double x = A[row * ld + i], y = A[row * ld + j];
                A[row * ld + i] = c * x - s * y;
                A[row * ld + j] = s * x + c * y;
                x = V[row * ld + i];
                y = V[row * ld + j];
                V[row * ld + i] = c * x - s * y;
                V[row * ld + j] = s * x + c * y;
            }
            __syncthreads();
            // round-robin: keep pos[0], rotate pos[1..pp-1] by one
            if (tid == 0) {
                int last = pos[pp - 1];
                for (int i = pp - 1; i > 1; --i) pos[i] = pos[i - 1];
                if (pp > 1) pos[1] = last;
            }
            __syncthreads();
        }
    }
    if (!converged && tid == 0) ffb_flag(status, FFB_ERR_NOT_CONVERGED);
    __syncthreads();
    // sort descending (rank by value, ties by index), sign-normalise, write
    const int o = off_[k];
    double *U = evecs + cov_off[k];
    for (int i = tid; i < p; i += nt) {
        double li = A[i * ld + i];
        int rank = 0;
        for (int j = 0; j < p; ++j) {
            double lj = A[j * ld + j];
            rank += (lj > li) || (lj == li && j < i);
        }
        // sign: largest |entry| (first on ties) positive
        int piv = 0;
        double best = -1.0;
        for (int q = 0; q < p; ++q) {
            double a = fabs(V[q * ld + i]);
            if (a > best) {
                best = a;
                piv = q;
            }
        }
        double sg = (V[piv * ld + i] < 0.0) ? -1.0 : 1.0;
        if (evals) evals[o + rank] = li;
        if (evecs)
            for (int q = 0; q < p; ++q) U[q * p + rank] = sg * V[q * ld + i];
    }
}

int ffb_launch_eig(ffb_plan_t p, cudaStream_t s) {
    if (p->pmax > EIG_MAXP) return FFB_ERR_UNSUPPORTED;
    const int pp = p->pmax + (p->pmax & 1);
    const bool vglobal = pp > EIG_VSHARED_MAXP;
    const bool aglobal = pp > EIG_ASHARED_MAXP;
    const int ldmax = pp + 1;
    if (vglobal && !p->d_eig_work) {
        int e = ffb_check_cuda(cudaMalloc(&p->d_eig_work, sizeof(double) * (size_t)(p->k_max + 1) *
                                                              (aglobal ? 2 : 1) * ldmax * ldmax));
        if (e) return e;
    }
    const size_t tail = sizeof(double) * ((size_t)pp + 256) + sizeof(int) * (size_t)(2 * pp);
    size_t smem = aglobal   ? tail
                  : vglobal ? sizeof(double) * (size_t)ldmax * ldmax + tail
                            : sizeof(double) * 2 * (size_t)pp * (pp + 1) + tail;
    static int attr = 0;
    if (smem > 48 * 1024 && attr < (int)smem) {
        int e = ffb_check_cuda(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (e) return e;
        attr = (int)smem;
    }
    ProfScope ps(p, FFB_KC_EIG, s);
    k_jacobi<<<p->k_max + 1, 256, smem, s>>>(p->d_Cfin, p->d_p, p->d_off, p->d_cov_off, p->d_evals, p->d_evecs,
                                             p->d_status, vglobal ? p->d_eig_work : nullptr, ldmax,
                                             aglobal ? 1 : 0);
    p->launches++;
    return ffb_check_cuda(cudaGetLastError());
}
