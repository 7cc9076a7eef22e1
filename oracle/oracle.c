/*
 * Oracle for the streaming, partitioned, randomized SVD of Maulik & Mengaldo,
 * "PyParSVD: A streaming, distributed and randomized singular-value-decomposition
 * library" (arXiv 2108.08845).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Plain, slow, obviously-correct FP64 CPU
 * code that runs the paper's algorithms step by step.  It shares no code, header,
 * table or helper with the CUDA library; only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline leg may load it.
 *
 * All matrices are column-major doubles: element (i, j) of an m x n matrix with
 * leading dimension ld is X[i + j*ld].  No blocking, fusion or reordering beyond
 * what the cited algorithm states; OpenMP only splits independent columns (or
 * rows) of one step across threads, each output being computed by one thread in a
 * fixed order, so results do not depend on the thread count.
 *
 * Contents (paper section / equation / algorithm each routine follows):
 *   orc_householder_qr   - the QR factorisation used in Algorithm 1 steps I1 and 1
 *                          (Householder reflections, Golub & Van Loan Alg. 5.2.1).
 *   orc_jacobi_svd       - the SVD of the small factor in Algorithm 1 steps I2 and 2
 *                          (one-sided Jacobi, Hestenes 1958).
 *   orc_stream_initialize, orc_stream_update
 *                        - Algorithm 1 (streaming SVD, Sec. 3.1).
 *   orc_tsqr_r           - the row-partitioned QR of Sec. 4.2 (local QR per block,
 *                          QR of the stacked R factors).
 *   orc_apmos            - Algorithm 2 (approximate partitioned method of
 *                          snapshots, Sec. 3.2).
 *   orc_rsvd_panel       - the randomized low-rank SVD of Sec. 3.3 applied to the
 *                          Algorithm 1 panel (range basis Q of P*Omega, optional
 *                          power iterations, SVD of Q^T P, U = Q U~).
 *   orc_philox4x32 / orc_philox4x64
 *                        - Philox4xW-10 counter-based generator (Salmon et al.,
 *                          SC'11), the Gaussian test matrix of Sec. 3.3.
 *   orc_gaussian         - Box-Muller (1958) transform with self-written log and
 *                          sin/cos series, bit-reproducible from IEEE +,*,/,fma,sqrt.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* Status codes (the oracle's own; independent of the library's). */
#define ORC_OK 0
#define ORC_ERR_SHAPE -1
#define ORC_ERR_NOT_CONVERGED -2
#define ORC_ERR_ALLOC -3

static double dot_col(int64_t len, const double* x, const double* y) {
  double s = 0.0;
  for (int64_t i = 0; i < len; ++i) s += x[i] * y[i];
  return s;
}

/* ------------------------------------------------------------------------- */
/* Householder QR (thin): A (m x n, m >= n) = Q (m x n) R (n x n, upper).     */
/* Reflector j maps column j (rows j..m-1) to alpha*e_j with                  */
/* alpha = -sign(x0)*||x||; v = x - alpha*e_1; H = I - beta v v^T,            */
/* beta = 2 / (v^T v).  Q = H_0 H_1 ... H_{n-1} [I_n; 0] by backward           */
/* accumulation.  Finally R's rows / Q's columns are flipped so that          */
/* diag(R) >= 0, which makes the factorisation unique for full-rank A.        */
/* A is overwritten.                                                          */
/* ------------------------------------------------------------------------- */
int orc_householder_qr(int64_t m, int64_t n, double* A, int64_t lda, double* Q, int64_t ldq,
                       double* R, int64_t ldr) {
  if (m < n || n < 0) return ORC_ERR_SHAPE;
  if (n == 0) return ORC_OK;
  double* V = (double*)calloc((size_t)m * (size_t)n, sizeof(double)); /* reflector j in column j */
  double* beta = (double*)calloc((size_t)n, sizeof(double));
  if (!V || !beta) {
    free(V);
    free(beta);
    return ORC_ERR_ALLOC;
  }
  for (int64_t j = 0; j < n; ++j) {
    const int64_t len = m - j;
    double* x = &A[IDX(j, j, lda)];
    double* v = &V[IDX(j, j, m)];
    double nrm2 = dot_col(len, x, x);
    double nrm = sqrt(nrm2);
    double alpha = (x[0] >= 0.0) ? -nrm : nrm;
    for (int64_t i = 0; i < len; ++i) v[i] = x[i];
    v[0] -= alpha;
    double vtv = dot_col(len, v, v);
    double b = (vtv > 0.0) ? 2.0 / vtv : 0.0;
    beta[j] = b;
    /* apply H_j to the trailing columns j+1..n-1 */
#pragma omp parallel for schedule(static)
    for (int64_t k = j + 1; k < n; ++k) {
      double* a = &A[IDX(j, k, lda)];
      double w = b * dot_col(len, v, a);
      for (int64_t i = 0; i < len; ++i) a[i] -= w * v[i];
    }
    /* column j becomes alpha * e_j */
    x[0] = (b > 0.0) ? alpha : x[0];
    for (int64_t i = 1; i < len; ++i) x[i] = (b > 0.0) ? 0.0 : x[i];
  }
  /* R = upper triangle of A(0:n, 0:n) */
  for (int64_t k = 0; k < n; ++k)
    for (int64_t i = 0; i < n; ++i) R[IDX(i, k, ldr)] = (i <= k) ? A[IDX(i, k, lda)] : 0.0;
  /* Q = H_0 ... H_{n-1} [I_n; 0], applied right to left */
  for (int64_t k = 0; k < n; ++k)
    for (int64_t i = 0; i < m; ++i) Q[IDX(i, k, ldq)] = (i == k) ? 1.0 : 0.0;
  for (int64_t j = n - 1; j >= 0; --j) {
    const int64_t len = m - j;
    const double* v = &V[IDX(j, j, m)];
    const double b = beta[j];
    if (b == 0.0) continue;
#pragma omp parallel for schedule(static)
    for (int64_t k = j; k < n; ++k) {
      double* q = &Q[IDX(j, k, ldq)];
      double w = b * dot_col(len, v, q);
      for (int64_t i = 0; i < len; ++i) q[i] -= w * v[i];
    }
  }
  /* sign normalisation: diag(R) >= 0 */
  for (int64_t i = 0; i < n; ++i) {
    if (R[IDX(i, i, ldr)] < 0.0) {
      for (int64_t k = i; k < n; ++k) R[IDX(i, k, ldr)] = -R[IDX(i, k, ldr)];
      for (int64_t r = 0; r < m; ++r) Q[IDX(r, i, ldq)] = -Q[IDX(r, i, ldq)];
    }
  }
  free(V);
  free(beta);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* One-sided Jacobi SVD (Hestenes).  W (m x n) is overwritten: on exit its    */
/* columns are mutually orthogonal, W = A V.  V (n x n) accumulates the       */
/* plane rotations (starts as I).  sigma_j = ||w_j||.  Pairs are visited in   */
/* cyclic-by-rows order (p < q).  A pair is rotated when                      */
/* |w_p^T w_q| > tol * ||w_p|| ||w_q||; the rotation angle zeroes the 2x2 Gram */
/* off-diagonal (t = sign(z)/(|z| + sqrt(1+z^2)), z = (b - a)/(2g)).          */
/* The sweep loop stops after a sweep with no rotation.  A column whose norm  */
/* is at most m*eps times the largest column norm (measured at the start of   */
/* the sweep) is treated as zero and not rotated, so rank-deficient inputs    */
/* terminate (their tail singular values are then noise of size m*eps*s_max). */
/* Returns the number of sweeps, or ORC_ERR_NOT_CONVERGED.                    */
/* ------------------------------------------------------------------------- */
int orc_jacobi_svd(int64_t m, int64_t n, double* W, int64_t ldw, double* V, int64_t ldv,
                   double* sigma, int max_sweeps, double tol) {
  for (int64_t k = 0; k < n; ++k)
    for (int64_t i = 0; i < n; ++i) V[IDX(i, k, ldv)] = (i == k) ? 1.0 : 0.0;
  int sweep = 0;
  int converged = (n <= 1);
  while (!converged && sweep < max_sweeps) {
    ++sweep;
    int rotated = 0;
    double cmax = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      const double* w = &W[IDX(0, k, ldw)];
      double a = dot_col(m, w, w);
      cmax = (a > cmax) ? a : cmax;
    }
    const double negl = (double)m * 2.220446049250313e-16;
    const double negl2 = negl * negl * cmax; /* (m eps max||w||)^2 */
    for (int64_t p = 0; p < n - 1; ++p) {
      for (int64_t q = p + 1; q < n; ++q) {
        double* wp = &W[IDX(0, p, ldw)];
        double* wq = &W[IDX(0, q, ldw)];
        double a = dot_col(m, wp, wp);
        double b = dot_col(m, wq, wq);
        double g = dot_col(m, wp, wq);
        if (a <= negl2 || b <= negl2) continue;
        if (!(fabs(g) > tol * sqrt(a) * sqrt(b))) continue;
        rotated = 1;
        double z = (b - a) / (2.0 * g);
        double t = ((z >= 0.0) ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = c * t;
        for (int64_t i = 0; i < m; ++i) {
          double xp = wp[i], xq = wq[i];
          wp[i] = c * xp - s * xq;
          wq[i] = s * xp + c * xq;
        }
        double* vp = &V[IDX(0, p, ldv)];
        double* vq = &V[IDX(0, q, ldv)];
        for (int64_t i = 0; i < n; ++i) {
          double xp = vp[i], xq = vq[i];
          vp[i] = c * xp - s * xq;
          vq[i] = s * xp + c * xq;
        }
      }
    }
    if (!rotated) converged = 1;
  }
  for (int64_t k = 0; k < n; ++k) {
    const double* w = &W[IDX(0, k, ldw)];
    sigma[k] = sqrt(dot_col(m, w, w));
  }
  return converged ? sweep : ORC_ERR_NOT_CONVERGED;
}

/* Stable descending order of sigma: order[0] is the index of the largest;
 * equal values keep their original (lower index first) order. */
void orc_sort_desc(int64_t n, const double* sigma, int64_t* order) {
  for (int64_t i = 0; i < n; ++i) order[i] = i;
  for (int64_t i = 1; i < n; ++i) { /* insertion sort: stable */
    int64_t cur = order[i];
    int64_t j = i - 1;
    while (j >= 0 && sigma[order[j]] < sigma[cur]) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = cur;
  }
}

/* SVD of a square n x n matrix R (Algorithm 1 steps I2 / 2): R = U~ D~ V~^T.
 * Jacobi on the columns of R gives R V~ = W, so U~ = W D~^{-1}.  Outputs are
 * sorted by descending singular value.  Uo, Vo: n x n (ld n); d: n.
 * A zero singular value leaves its U~ column zero. */
static int svd_square(int64_t n, const double* R, int64_t ldr, double* Uo, double* d, double* Vo,
                      int max_sweeps, double tol) {
  double* W = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!W || !V || !s || !order) {
    free(W); free(V); free(s); free(order);
    return ORC_ERR_ALLOC;
  }
  for (int64_t k = 0; k < n; ++k)
    for (int64_t i = 0; i < n; ++i) W[IDX(i, k, n)] = R[IDX(i, k, ldr)];
  int rc = orc_jacobi_svd(n, n, W, n, V, n, s, max_sweeps, tol);
  orc_sort_desc(n, s, order);
  for (int64_t k = 0; k < n; ++k) {
    int64_t src = order[k];
    d[k] = s[src];
    for (int64_t i = 0; i < n; ++i) {
      Uo[IDX(i, k, n)] = (s[src] > 0.0) ? W[IDX(i, src, n)] / s[src] : 0.0;
      Vo[IDX(i, k, n)] = V[IDX(i, src, n)];
    }
  }
  free(W); free(V); free(s); free(order);
  return rc < 0 ? rc : ORC_OK;
}

/* C (m x k) = A (m x n) * B (n x k), rows split across threads. */
static void matmul(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                   int64_t ldb, double* C, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t c = 0; c < k; ++c) {
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s += A[IDX(i, j, lda)] * B[IDX(j, c, ldb)];
      C[IDX(i, c, ldc)] = s;
    }
  }
}

/* C (n x k) = A^T (n x m) * B (m x k): each entry a dot product over rows. */
static void matmul_tn(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda,
                      const double* B, int64_t ldb, double* C, int64_t ldc) {
#pragma omp parallel for schedule(static) collapse(2)
  for (int64_t c = 0; c < k; ++c)
    for (int64_t j = 0; j < n; ++j) C[IDX(j, c, ldc)] = dot_col(m, &A[IDX(0, j, lda)], &B[IDX(0, c, ldb)]);
}

/* The QR + small SVD + truncation shared by Algorithm 1's initialisation (I1-I2)
 * and its update (steps 1-5): P (m x n) = Q R; R = U~ D~ V~^T (sorted);
 * U = Q U~(:, 0:K); D = D~(0:K).  P is overwritten. */
static int qr_svd_truncate(int64_t m, int64_t n, int64_t K, double* P, int64_t ldp, double* U,
                           int64_t ldu, double* D, int max_sweeps, double tol) {
  if (m < n || K > n) return ORC_ERR_SHAPE;
  double* Q = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
  double* R = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* Ut = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* Vt = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  if (!Q || !R || !Ut || !Vt || !d) {
    free(Q); free(R); free(Ut); free(Vt); free(d);
    return ORC_ERR_ALLOC;
  }
  int rc = orc_householder_qr(m, n, P, ldp, Q, m, R, n);
  if (rc == ORC_OK) rc = svd_square(n, R, n, Ut, d, Vt, max_sweeps, tol);
  if (rc == ORC_OK) {
    matmul(m, n, K, Q, m, Ut, n, U, ldu); /* U = Q U~_K */
    for (int64_t k = 0; k < K; ++k) D[k] = d[k];
  }
  free(Q); free(R); free(Ut); free(Vt); free(d);
  return rc;
}

/* Algorithm 1, initialisation I1-I2: A0 (m x B) = Q R; R = U' D0 V0^T;
 * U0 = Q U' truncated to k0 = min(K, B) columns (the slice [:, :K] of a B-column
 * matrix), D0 truncated likewise.  Requires B <= m.  U: m x k0 (ldu), D: k0.
 * A0 is not modified.  Returns k0 (> 0) or a negative status. */
int orc_stream_initialize(int64_t m, int64_t B, int64_t K, const double* A0, int64_t lda,
                          double* U, int64_t ldu, double* D, int max_sweeps, double tol) {
  if (B > m || K < 1 || B < 1) return ORC_ERR_SHAPE;
  const int64_t k0 = (K < B) ? K : B;
  double* P = (double*)malloc(sizeof(double) * (size_t)m * (size_t)B);
  if (!P) return ORC_ERR_ALLOC;
  for (int64_t j = 0; j < B; ++j) memcpy(&P[IDX(0, j, m)], &A0[IDX(0, j, lda)], sizeof(double) * (size_t)m);
  int rc = qr_svd_truncate(m, B, k0, P, m, U, ldu, D, max_sweeps, tol);
  free(P);
  return rc < 0 ? rc : (int)k0;
}

/* Algorithm 1, steps 1-5 for one new batch A (m x B), with kc current modes:
 *   1. QR of the column-wise concatenation [ff * U * diag(D) | A]   (m x (kc+B))
 *   2. SVD of its R factor
 *   3./5. keep the first k1 = min(K, kc+B) singular vectors / values (descending)
 *   4. U <- Q * U~_k1
 * U (m x K buffer, ldu; first kc columns valid) and D (K) are updated in place.
 * Returns k1 (> 0) or a negative status. */
int orc_stream_update(int64_t m, int64_t kc, int64_t K, int64_t B, double ff, double* U,
                      int64_t ldu, double* D, const double* A, int64_t lda, int max_sweeps,
                      double tol) {
  const int64_t n = kc + B;
  if (m < n || kc < 0 || kc > K || B < 1) return ORC_ERR_SHAPE;
  const int64_t k1 = (K < n) ? K : n;
  double* P = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
  if (!P) return ORC_ERR_ALLOC;
  for (int64_t j = 0; j < kc; ++j) {
    const double scale = ff * D[j];
    for (int64_t i = 0; i < m; ++i) P[IDX(i, j, m)] = scale * U[IDX(i, j, ldu)];
  }
  for (int64_t j = 0; j < B; ++j) memcpy(&P[IDX(0, kc + j, m)], &A[IDX(0, j, lda)], sizeof(double) * (size_t)m);
  int rc = qr_svd_truncate(m, n, k1, P, m, U, ldu, D, max_sweeps, tol);
  free(P);
  return rc < 0 ? rc : (int)k1;
}

/* Row-partitioned QR (Sec. 4.2, the parallel QR used by the streaming update):
 * each row block [off[b], off[b+1]) of A (m x n) is QR-factored locally; the
 * local R factors are stacked (nparts*n x n) and QR-factored again; the result R
 * (n x n, diag >= 0) is written to Rout.  Every block needs >= n rows. */
int orc_tsqr_r(int64_t m, int64_t n, const double* A, int64_t lda, int64_t nparts,
               const int64_t* off, double* Rout, int64_t ldr) {
  if (nparts < 1 || off[0] != 0 || off[nparts] != m) return ORC_ERR_SHAPE;
  for (int64_t b = 0; b < nparts; ++b)
    if (off[b + 1] - off[b] < n) return ORC_ERR_SHAPE;
  const int64_t ms = nparts * n;
  double* S = (double*)malloc(sizeof(double) * (size_t)ms * (size_t)n);
  double* Qs = (double*)malloc(sizeof(double) * (size_t)ms * (size_t)n);
  if (!S || !Qs) { free(S); free(Qs); return ORC_ERR_ALLOC; }
  int rc = ORC_OK;
  for (int64_t b = 0; b < nparts && rc == ORC_OK; ++b) {
    const int64_t mb = off[b + 1] - off[b];
    double* Ab = (double*)malloc(sizeof(double) * (size_t)mb * (size_t)n);
    double* Qb = (double*)malloc(sizeof(double) * (size_t)mb * (size_t)n);
    double* Rb = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    if (!Ab || !Qb || !Rb) rc = ORC_ERR_ALLOC;
    if (rc == ORC_OK) {
      for (int64_t j = 0; j < n; ++j)
        memcpy(&Ab[IDX(0, j, mb)], &A[IDX(off[b], j, lda)], sizeof(double) * (size_t)mb);
      rc = orc_householder_qr(mb, n, Ab, mb, Qb, mb, Rb, n);
      for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) S[IDX(b * n + i, j, ms)] = Rb[IDX(i, j, n)];
    }
    free(Ab); free(Qb); free(Rb);
  }
  if (rc == ORC_OK) rc = orc_householder_qr(ms, n, S, ms, Qs, ms, Rout, ldr);
  free(S); free(Qs);
  return rc;
}

/* Algorithm 2 (APMOS).  A (m x N) is split into row blocks [off[b], off[b+1]).
 *  1. local SVD of each block: A^b = Q R (Householder), R = U~ S V^T (Jacobi);
 *     the block's right singular vectors are V, its singular values S.
 *  2. keep r1 columns: V~^b = V(:, 0:r1), S~^b = S(0:r1).
 *  3. W = [V~^1 S~^1, ..., V~^nb S~^nb]  (N x r1*nb).
 *  4. SVD of W = X L Y^T: one-sided Jacobi on the columns of W^T gives
 *     W^T V' = Z with orthogonal columns, hence X = V' and L = ||z_j||.
 *  5. keep r2 columns of X and values of L.
 *  7. U~^b_j = A^b X~_j / L~_j for every block b and kept column j.
 * Uout: m x r2 (ldu), Lout: r2.  Every block needs >= N rows. */
int orc_apmos(int64_t m, int64_t N, const double* A, int64_t lda, int64_t nparts,
              const int64_t* off, int64_t r1, int64_t r2, double* Uout, int64_t ldu, double* Lout,
              int max_sweeps, double tol) {
  if (nparts < 1 || off[0] != 0 || off[nparts] != m || r1 < 1 || r1 > N || r2 < 1) return ORC_ERR_SHAPE;
  for (int64_t b = 0; b < nparts; ++b)
    if (off[b + 1] - off[b] < N) return ORC_ERR_SHAPE;
  const int64_t wc = r1 * nparts; /* columns of W */
  if (r2 > N || r2 > wc) return ORC_ERR_SHAPE;
  double* Wt = (double*)calloc((size_t)wc * (size_t)N, sizeof(double)); /* W^T: wc x N */
  int rc = Wt ? ORC_OK : ORC_ERR_ALLOC;
  for (int64_t b = 0; b < nparts && rc == ORC_OK; ++b) {
    const int64_t mb = off[b + 1] - off[b];
    double* Ab = (double*)malloc(sizeof(double) * (size_t)mb * (size_t)N);
    double* Qb = (double*)malloc(sizeof(double) * (size_t)mb * (size_t)N);
    double* Rb = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N);
    double* Ub = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N);
    double* Vb = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N);
    double* sb = (double*)malloc(sizeof(double) * (size_t)N);
    if (!Ab || !Qb || !Rb || !Ub || !Vb || !sb) rc = ORC_ERR_ALLOC;
    if (rc == ORC_OK) {
      for (int64_t j = 0; j < N; ++j)
        memcpy(&Ab[IDX(0, j, mb)], &A[IDX(off[b], j, lda)], sizeof(double) * (size_t)mb);
      rc = orc_householder_qr(mb, N, Ab, mb, Qb, mb, Rb, N);
      if (rc == ORC_OK) rc = svd_square(N, Rb, N, Ub, sb, Vb, max_sweeps, tol);
      /* W block b = V~^b S~^b ; stored transposed: row (b*r1 + k) of W^T */
      for (int64_t k = 0; k < r1 && rc == ORC_OK; ++k)
        for (int64_t i = 0; i < N; ++i) Wt[IDX(b * r1 + k, i, wc)] = Vb[IDX(i, k, N)] * sb[k];
    }
    free(Ab); free(Qb); free(Rb); free(Ub); free(Vb); free(sb);
  }
  if (rc != ORC_OK) { free(Wt); return rc; }
  double* Vp = (double*)malloc(sizeof(double) * (size_t)N * (size_t)N);
  double* lam = (double*)malloc(sizeof(double) * (size_t)N);
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  double* Xt = (double*)malloc(sizeof(double) * (size_t)N * (size_t)r2);
  if (!Vp || !lam || !order || !Xt) rc = ORC_ERR_ALLOC;
  if (rc == ORC_OK) {
    int s = orc_jacobi_svd(wc, N, Wt, wc, Vp, N, lam, max_sweeps, tol);
    if (s < 0) rc = s;
    orc_sort_desc(N, lam, order);
    for (int64_t j = 0; j < r2; ++j) {
      const int64_t src = order[j];
      Lout[j] = lam[src];
      const double inv = (lam[src] > 0.0) ? 1.0 / lam[src] : 0.0; /* L_j = 0: mode set to zero */
      for (int64_t i = 0; i < N; ++i) Xt[IDX(i, j, N)] = Vp[IDX(i, src, N)] * inv;
    }
    matmul(m, N, r2, A, lda, Xt, N, Uout, ldu); /* every block: A^b X~_j / L~_j */
  }
  free(Wt); free(Vp); free(lam); free(order); free(Xt);
  return rc;
}

/* Q factor of a thin Householder QR (m x n), returned in Y's place. */
static int orthonormalise(int64_t m, int64_t n, double* Y, int64_t ldy) {
  double* Q = (double*)malloc(sizeof(double) * (size_t)m * (size_t)n);
  double* R = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!Q || !R) { free(Q); free(R); return ORC_ERR_ALLOC; }
  int rc = orc_householder_qr(m, n, Y, ldy, Q, m, R, n);
  for (int64_t j = 0; j < n; ++j) memcpy(&Y[IDX(0, j, ldy)], &Q[IDX(0, j, m)], sizeof(double) * (size_t)m);
  free(Q); free(R);
  return rc;
}

/* Randomized low-rank SVD (Sec. 3.3) of the panel P (m x n) to rank K, with the
 * range basis built as in Halko, Martinsson & Tropp (2011) randomized subspace
 * iteration: Y = P Omega (Omega: n x l Gaussian), Q = orth(Y); q times:
 * Q^ = orth(P^T Q), Q = orth(P Q^).  Then Bm = Q^T P (l x n), SVD of Bm by
 * Jacobi on the columns of Bm^T (Bm^T V' = Z, so U~ = V'), sorted, and
 * U = Q U~_K, D = sigma_K.  The sign of each kept mode u_j is fixed so that
 * (P 1)^T u_j >= 0 (the paper leaves signs free; with a fixed Omega the next
 * randomized update depends on them, so a convention makes the streamed result
 * a function of the data and the seed alone).  P is not modified.  Requires
 * K <= l <= n <= m. */
int orc_rsvd_panel(int64_t m, int64_t n, const double* P, int64_t ldp, int64_t K, int64_t l,
                   const double* Omega, int64_t ldo, int64_t q, double* U, int64_t ldu, double* D,
                   int max_sweeps, double tol) {
  if (K < 1 || K > l || l > n || n > m) return ORC_ERR_SHAPE;
  double* Y = (double*)malloc(sizeof(double) * (size_t)m * (size_t)l);
  double* Z = (double*)malloc(sizeof(double) * (size_t)n * (size_t)l);
  double* Bt = (double*)malloc(sizeof(double) * (size_t)n * (size_t)l);
  double* Vp = (double*)malloc(sizeof(double) * (size_t)l * (size_t)l);
  double* s = (double*)malloc(sizeof(double) * (size_t)l);
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)l);
  double* Uk = (double*)malloc(sizeof(double) * (size_t)l * (size_t)K);
  int rc = (Y && Z && Bt && Vp && s && order && Uk) ? ORC_OK : ORC_ERR_ALLOC;
  if (rc == ORC_OK) {
    matmul(m, n, l, P, ldp, Omega, ldo, Y, m); /* Y = P Omega */
    rc = orthonormalise(m, l, Y, m);
  }
  for (int64_t it = 0; it < q && rc == ORC_OK; ++it) {
    matmul_tn(m, n, l, P, ldp, Y, m, Z, n); /* Z = P^T Q */
    rc = orthonormalise(n, l, Z, n);
    if (rc == ORC_OK) {
      matmul(m, n, l, P, ldp, Z, n, Y, m); /* Y = P Q^ */
      rc = orthonormalise(m, l, Y, m);
    }
  }
  if (rc == ORC_OK) {
    matmul_tn(m, n, l, P, ldp, Y, m, Bt, n); /* Bm^T = P^T Q  (n x l) */
    int sw = orc_jacobi_svd(n, l, Bt, n, Vp, l, s, max_sweeps, tol);
    if (sw < 0) rc = sw;
    orc_sort_desc(l, s, order);
    for (int64_t j = 0; j < K; ++j) {
      D[j] = s[order[j]];
      for (int64_t i = 0; i < l; ++i) Uk[IDX(i, j, l)] = Vp[IDX(i, order[j], l)];
    }
    matmul(m, l, K, Y, m, Uk, l, U, ldu); /* U = Q U~_K */
    /* sign convention: (P 1)^T u_j >= 0 for every kept mode j (Y reused for P 1) */
    for (int64_t i = 0; i < m; ++i) {
      double rowsum = 0.0;
      for (int64_t c = 0; c < n; ++c) rowsum += P[IDX(i, c, ldp)];
      Y[i] = rowsum;
    }
    for (int64_t j = 0; j < K; ++j) {
      if (dot_col(m, Y, &U[IDX(0, j, ldu)]) < 0.0)
        for (int64_t i = 0; i < m; ++i) U[IDX(i, j, ldu)] = -U[IDX(i, j, ldu)];
    }
  }
  free(Y); free(Z); free(Bt); free(Vp); free(s); free(order); free(Uk);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Philox4xW-R (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as     */
/* easy as 1, 2, 3", SC'11).  One round on counter (x0,x1,x2,x3), key (k0,k1):*/
/*   (h0,l0) = mulhilo(M0, x0); (h1,l1) = mulhilo(M1, x2)                     */
/*   x <- (h1 ^ x1 ^ k0, l1, h0 ^ x3 ^ k1, l0)                                 */
/* and the key is bumped by the Weyl constants (W0, W1) between rounds.       */
/* ------------------------------------------------------------------------- */
static const uint32_t PH32_M0 = 0xD2511F53u, PH32_M1 = 0xCD9E8D57u;
static const uint32_t PH32_W0 = 0x9E3779B9u, PH32_W1 = 0xBB67AE85u;
static const uint64_t PH64_M0 = 0xD2E7470EE14C6C93ull, PH64_M1 = 0xCA5A826395121157ull;
static const uint64_t PH64_W0 = 0x9E3779B97F4A7C15ull, PH64_W1 = 0xBB67AE8584CAA73Bull;

void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], int rounds, uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < rounds; ++r) {
    if (r > 0) {
      k0 += PH32_W0;
      k1 += PH32_W1;
    }
    uint64_t p0 = (uint64_t)PH32_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PH32_M1 * (uint64_t)x2;
    uint32_t h0 = (uint32_t)(p0 >> 32), l0 = (uint32_t)p0;
    uint32_t h1 = (uint32_t)(p1 >> 32), l1 = (uint32_t)p1;
    uint32_t y0 = h1 ^ x1 ^ k0, y1 = l1, y2 = h0 ^ x3 ^ k1, y3 = l0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  /* schoolbook 32-bit limbs: exact 128-bit product */
  uint64_t a0 = a & 0xffffffffull, a1 = a >> 32, b0 = b & 0xffffffffull, b1 = b >> 32;
  uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
  uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffull) + (p10 & 0xffffffffull);
  *lo = (p00 & 0xffffffffull) | (mid << 32);
  *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], int rounds, uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < rounds; ++r) {
    if (r > 0) {
      k0 += PH64_W0;
      k1 += PH64_W1;
    }
    uint64_t h0, l0, h1, l1;
    mulhilo64(PH64_M0, x0, &h0, &l0);
    mulhilo64(PH64_M1, x2, &h1, &l1);
    uint64_t y0 = h1 ^ x1 ^ k0, y1 = l1, y2 = h0 ^ x3 ^ k1, y3 = l0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------- */
/* Gaussian transform.  Built only from IEEE-754 binary64 operations that are */
/* correctly rounded everywhere (+, -, *, /, sqrt, fma), evaluated in a fixed */
/* order, so any implementation that performs the same operations produces    */
/* the same bits.  This file is compiled with -ffp-contract=off.              */
/*                                                                            */
/* ln(x), x in (0, 1]:  x = m 2^e with m in [sqrt(1/2), sqrt(2)];             */
/*   ln(m) = 2 atanh(s) = 2 s sum_{k>=0} s^{2k}/(2k+1),  s = (m-1)/(m+1),     */
/*   |s| <= 0.1716, 13 terms (truncation < 1e-20); ln(x) = e ln2 + ln(m).     */
/* sin, cos of theta = 2 pi u, u in [0, 1): quadrant q = floor(4u),           */
/*   phi = (4u - q) pi/2 in [0, pi/2); Taylor series of sin(phi), cos(phi)    */
/*   through phi^25 and phi^24 (truncation < 1e-20); rotate by q quadrants.   */
/* Box-Muller (1958): r = sqrt(-2 ln u1), z0 = r cos(theta), z1 = r sin(theta).*/
/* ------------------------------------------------------------------------- */
/* 1/(2k+1), k = 0..12, as exactly-rounded binary64 literals */
static const double ATANH_C[13] = {
    0x1p+0,
    0x1.5555555555555p-2,
    0x1.999999999999ap-3,
    0x1.2492492492492p-3,
    0x1.c71c71c71c71cp-4,
    0x1.745d1745d1746p-4,
    0x1.3b13b13b13b14p-4,
    0x1.1111111111111p-4,
    0x1.e1e1e1e1e1e1ep-5,
    0x1.af286bca1af28p-5,
    0x1.8618618618618p-5,
    0x1.642c8590b2164p-5,
    0x1.47ae147ae147bp-5,
};
/* (-1)^k / (2k+1)!, k = 0..12 (sin) and (-1)^k / (2k)!, k = 0..12 (cos) */
static const double SIN_C[13] = {
    0x1p+0,
    -0x1.5555555555555p-3,
    0x1.1111111111111p-7,
    -0x1.a01a01a01a01ap-13,
    0x1.71de3a556c734p-19,
    -0x1.ae64567f544e4p-26,
    0x1.6124613a86d09p-33,
    -0x1.ae7f3e733b81fp-41,
    0x1.952c77030ad4ap-49,
    -0x1.2f49b46814157p-57,
    0x1.71b8ef6dcf572p-66,
    -0x1.761b41316381ap-75,
    0x1.3f3ccdd165fa9p-84,
};
static const double COS_C[13] = {
    0x1p+0,
    -0x1p-1,
    0x1.5555555555555p-5,
    -0x1.6c16c16c16c17p-10,
    0x1.a01a01a01a01ap-16,
    -0x1.27e4fb7789f5cp-22,
    0x1.1eed8eff8d898p-29,
    -0x1.93974a8c07c9dp-37,
    0x1.ae7f3e733b81fp-45,
    -0x1.6827863b97d97p-53,
    0x1.e542ba4020225p-62,
    -0x1.0ce396db7f853p-70,
    0x1.f2cf01972f578p-80,
};
static const double LN2 = 0x1.62e42fefa39efp-1;
static const double PI_2 = 0x1.921fb54442d18p+0;
static const double SQRT1_2 = 0x1.6a09e667f3bcdp-1;

double orc_ln(double x) {
  uint64_t bits;
  memcpy(&bits, &x, 8);
  int64_t e = (int64_t)((bits >> 52) & 0x7ff) - 1023;
  uint64_t mb = (bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
  double m;
  memcpy(&m, &mb, 8); /* m in [1, 2) */
  if (m > 2.0 * SQRT1_2) {
    m = m * 0.5;
    e += 1;
  }
  double s = (m - 1.0) / (m + 1.0);
  double z = s * s;
  double p = ATANH_C[12];
  for (int k = 11; k >= 0; --k) p = fma(p, z, ATANH_C[k]);
  double lnm = (2.0 * s) * p;
  return fma((double)e, LN2, lnm);
}

void orc_sincos_2pi(double u, double* sn, double* cs) {
  double u4 = 4.0 * u;
  double qd = floor(u4);
  int q = (int)qd;
  double phi = (u4 - qd) * PI_2;
  double z = phi * phi;
  double ps = SIN_C[12], pc = COS_C[12];
  for (int k = 11; k >= 0; --k) {
    ps = fma(ps, z, SIN_C[k]);
    pc = fma(pc, z, COS_C[k]);
  }
  double s = phi * ps, c = pc;
  switch (q & 3) {
    case 0: *sn = s; *cs = c; break;
    case 1: *sn = c; *cs = -s; break;
    case 2: *sn = -s; *cs = -c; break;
    default: *sn = -c; *cs = s; break;
  }
}

/* 53-bit uniform in [0, 1) from two 32-bit words: (a>>5)*2^26 + (b>>6), over 2^53. */
static double uniform53(uint32_t a, uint32_t b) {
  uint64_t v = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
  return (double)v * 0x1p-53;
}

/* Gaussian variate number `idx` of stream (seed, stream): Philox4x32-10 on
 * counter (idx/2 low, idx/2 high, stream low, stream high), key (seed low,
 * seed high); u1 = 1 - uniform53(w0, w1) in (0, 1], u2 = uniform53(w2, w3);
 * even idx -> r cos(2 pi u2), odd idx -> r sin(2 pi u2). */
double orc_gaussian_one(uint64_t seed, uint64_t stream, uint64_t idx) {
  uint64_t pair = idx >> 1;
  uint32_t ctr[4] = {(uint32_t)pair, (uint32_t)(pair >> 32), (uint32_t)stream, (uint32_t)(stream >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32(ctr, key, 10, w);
  double u1 = 1.0 - uniform53(w[0], w[1]);
  double u2 = uniform53(w[2], w[3]);
  double r = sqrt(-2.0 * orc_ln(u1));
  double sn, cs;
  orc_sincos_2pi(u2, &sn, &cs);
  return (idx & 1) ? r * sn : r * cs;
}

/* Fills out[0..count) with Gaussian variates first_idx, first_idx+1, ... */
void orc_gaussian(uint64_t seed, uint64_t stream, uint64_t first_idx, int64_t count, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) out[i] = orc_gaussian_one(seed, stream, first_idx + (uint64_t)i);
}
