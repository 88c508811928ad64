/*
 * Type-generic body of the CPU oracle. Included twice by tbbt_oracle.c, once
 * with SCALAR = double (real symmetric problems) and once with
 * SCALAR = double complex (Hermitian problems). TEST INFRASTRUCTURE ONLY.
 *
 * Required macros: SCALAR, SFX (name suffix), CONJ(x), RE(x), IM(x),
 * IS_COMPLEX (0/1).
 */

#define CAT_(a, b) a##b
#define CAT(a, b) CAT_(a, b)
#define FN(name) CAT(name, SFX)

/*
 * Working storage of the band matrix during the reduction: lower triangle
 * only, W[(r - c) + c * ldw] = B[r][c] for 0 <= r - c <= 2b. The reduction
 * creates bulges of at most 2b - 1 sub-diagonals (the fill of a b x b block
 * placed b rows below the diagonal), so 2b + 1 diagonals always suffice.
 */
typedef struct {
  SCALAR *w;
  int64_t n, b, ldw;
} FN(band_t);

static SCALAR *FN(bat)(FN(band_t) * B, int64_t r, int64_t c) {
  if (!(r >= c && r - c <= 2 * B->b && r < B->n && c >= 0)) {
    fprintf(stderr, "oracle: band access out of range (%lld,%lld)\n", (long long)r, (long long)c);
    abort();
  }
  return &B->w[(r - c) + c * B->ldw];
}

/* Element (r, c) of the full Hermitian matrix. */
static SCALAR FN(bget)(FN(band_t) * B, int64_t r, int64_t c) {
  if (r >= c) return *FN(bat)(B, r, c);
  return CONJ(*FN(bat)(B, c, r));
}

/*
 * Householder generation (the "standard Householder method" cited with Eq. 7,
 * in the LAPACK convention): for x of length L find beta (real), tau and v
 * with v[0] = 1 such that H^H x = beta e_1, H = I - tau v v^H. If x[1:] = 0
 * and x[0] is real the reflector is the identity (tau = 0).
 */
static void FN(house)(int64_t L, const SCALAR *x, SCALAR *v, SCALAR *tau, double *beta) {
  SCALAR alpha = x[0];
  double s2 = 0.0;
  for (int64_t t = 1; t < L; ++t) s2 += RE(x[t]) * RE(x[t]) + IM(x[t]) * IM(x[t]);
  v[0] = 1.0;
  if (s2 == 0.0 && IM(alpha) == 0.0) {
    *tau = 0.0;
    *beta = RE(alpha);
    for (int64_t t = 1; t < L; ++t) v[t] = 0.0;
    return;
  }
  double a2 = RE(alpha) * RE(alpha) + IM(alpha) * IM(alpha);
  double nrm = sqrt(a2 + s2);
  double bt = RE(alpha) >= 0.0 ? -nrm : nrm;
  *beta = bt;
  *tau = (bt - alpha) / bt;
  SCALAR scal = 1.0 / (alpha - bt);
  for (int64_t t = 1; t < L; ++t) v[t] = x[t] * scal;
}

/*
 * Band -> tridiagonal reduction by bulge chasing (Eq. 6b, Sec. 2.2.1,
 * Fig. 2). Stage i (0-based, i = 0..n-3) has ceil((n-i-2)/b) sweeps; sweep j
 * works on rows r = i+1+j*b .. r+L-1 with L = min(b, n-r). Sweep 0 reduces
 * column i; sweep j >= 1 eliminates the first column (r-b) of the bulge made
 * by sweep j-1. Every transformation is applied two-sided (B <- H^H B H).
 * Hermitian problems get one more stage, i = n-2, whose length-1 reflector
 * makes the last sub-diagonal entry real.
 *
 * band:   lower band storage (b+1) x n, band[d + c*ldb] = B[c+d][c].
 * hh_v:   out, K x b column-major, reflector k at hh_v[k*b .. k*b+b), v[0]=1
 *         stored, zero beyond its length. hh_tau: out, K.
 * d, e:   out, diagonal (n) and real sub-diagonal (n-1) of T.
 * bandout (optional): the reduced working storage, (2b+1) x n, to check that
 *         everything beyond the first sub-diagonal is exactly zero.
 * Returns the number of reflectors written.
 */
int64_t FN(orc_bulge_chase_)(int64_t n, int64_t b, const SCALAR *band, int64_t ldb, SCALAR *hh_v,
                             SCALAR *hh_tau, double *d, double *e, SCALAR *bandout) {
  FN(band_t) B;
  B.n = n;
  B.b = b;
  B.ldw = 2 * b + 1;
  B.w = (SCALAR *)calloc((size_t)(B.ldw * (n > 0 ? n : 1)), sizeof(SCALAR));
  for (int64_t c = 0; c < n; ++c)
    for (int64_t dd = 0; dd <= b && c + dd < n; ++dd) B.w[dd + c * B.ldw] = band[dd + c * ldb];
  for (int64_t c = 0; c < n; ++c) B.w[c * B.ldw] = RE(B.w[c * B.ldw]); /* Hermitian diagonal */

  SCALAR *x = (SCALAR *)malloc(sizeof(SCALAR) * (size_t)(b + 1));
  SCALAR *v = (SCALAR *)malloc(sizeof(SCALAR) * (size_t)(b + 1));
  SCALAR *D = (SCALAR *)malloc(sizeof(SCALAR) * (size_t)((b + 1) * (b + 1)));
  SCALAR *y = (SCALAR *)malloc(sizeof(SCALAR) * (size_t)(b + 1));
  int64_t k = 0;
  int64_t last_stage = IS_COMPLEX ? n - 2 : n - 3;
  for (int64_t i = 0; i <= last_stage; ++i) {
    int64_t nsweep = (i <= n - 3) ? (n - i - 2 + b - 1) / b : 1;
    for (int64_t j = 0; j < nsweep; ++j) {
      int64_t r = i + 1 + j * b;
      int64_t L = (n - r < b) ? n - r : b;
      int64_t c = (j == 0) ? i : r - b;
      for (int64_t t = 0; t < L; ++t) x[t] = *FN(bat)(&B, r + t, c);
      SCALAR tau;
      double beta;
      FN(house)(L, x, v, &tau, &beta);
      *FN(bat)(&B, r, c) = beta;
      for (int64_t t = 1; t < L; ++t) *FN(bat)(&B, r + t, c) = 0.0;

      /* left: rows [r, r+L), columns c+1 .. r-1:  A <- H^H A */
      for (int64_t col = c + 1; col < r; ++col) {
        SCALAR w = 0.0;
        for (int64_t t = 0; t < L; ++t) w += CONJ(v[t]) * *FN(bat)(&B, r + t, col);
        for (int64_t t = 0; t < L; ++t) *FN(bat)(&B, r + t, col) -= CONJ(tau) * v[t] * w;
      }
      /* two-sided on the diagonal block [r, r+L)^2:  D <- H^H D H */
      for (int64_t s = 0; s < L; ++s)
        for (int64_t t = 0; t < L; ++t) D[t + s * L] = FN(bget)(&B, r + t, r + s);
      for (int64_t t = 0; t < L; ++t) { /* D <- D H : y = D v, D -= tau y v^H */
        SCALAR acc = 0.0;
        for (int64_t s = 0; s < L; ++s) acc += D[t + s * L] * v[s];
        y[t] = acc;
      }
      for (int64_t s = 0; s < L; ++s)
        for (int64_t t = 0; t < L; ++t) D[t + s * L] -= tau * y[t] * CONJ(v[s]);
      for (int64_t s = 0; s < L; ++s) { /* D <- H^H D : y = v^H D, D -= conj(tau) v y */
        SCALAR acc = 0.0;
        for (int64_t t = 0; t < L; ++t) acc += CONJ(v[t]) * D[t + s * L];
        y[s] = acc;
      }
      for (int64_t s = 0; s < L; ++s)
        for (int64_t t = 0; t < L; ++t) D[t + s * L] -= CONJ(tau) * v[t] * y[s];
      for (int64_t s = 0; s < L; ++s)
        for (int64_t t = s; t < L; ++t) *FN(bat)(&B, r + t, r + s) = D[t + s * L];
      for (int64_t s = 0; s < L; ++s) *FN(bat)(&B, r + s, r + s) = RE(D[s + s * L]);

      /* right: rows [r+L, min(r+L+b, n)), columns [r, r+L):  A <- A H */
      int64_t rend = (r + L + b < n) ? r + L + b : n;
      for (int64_t row = r + L; row < rend; ++row) {
        SCALAR w = 0.0;
        for (int64_t t = 0; t < L; ++t) w += *FN(bat)(&B, row, r + t) * v[t];
        for (int64_t t = 0; t < L; ++t) *FN(bat)(&B, row, r + t) -= tau * w * CONJ(v[t]);
      }
      if (hh_v) {
        for (int64_t t = 0; t < b; ++t) hh_v[k * b + t] = (t < L) ? v[t] : 0.0;
        hh_tau[k] = tau;
      }
      ++k;
    }
  }
  for (int64_t c = 0; c < n; ++c) {
    if (d) d[c] = RE(B.w[c * B.ldw]);
    if (e && c + 1 < n) {
      SCALAR sub = B.w[1 + c * B.ldw];
      if (IM(sub) != 0.0) {
        fprintf(stderr, "oracle: sub-diagonal %lld not real after reduction\n", (long long)c);
        abort();
      }
      e[c] = RE(sub);
    }
  }
  if (bandout) memcpy(bandout, B.w, sizeof(SCALAR) * (size_t)(B.ldw * n));
  free(x);
  free(v);
  free(D);
  free(y);
  free(B.w);
  return k;
}

/*
 * Tridiagonal -> band back-transformation of eigenvectors, Eq. 6d:
 * Z = H_0 H_1 ... H_{K-1} X, each H_k = I - tau_k v_k v_k^H applied as in
 * Eq. 8, x <- x - tau v (v^H x), in exact reverse generation order
 * (Sec. 2.2.2). Columns are independent, so threads take column blocks.
 */
typedef struct {
  int64_t n, b, K, c0, c1, ldq;
  const SCALAR *v;
  const SCALAR *tau;
  const int64_t *r;
  const int64_t *L;
  SCALAR *q;
} FN(bt_job_t);

static void *FN(bt_worker)(void *arg) {
  FN(bt_job_t) *J = (FN(bt_job_t) *)arg;
  for (int64_t k = J->K - 1; k >= 0; --k) {
    const SCALAR *vk = J->v + k * J->b;
    SCALAR tk = J->tau[k];
    int64_t r = J->r[k], L = J->L[k];
    for (int64_t c = J->c0; c < J->c1; ++c) {
      SCALAR *x = J->q + c * J->ldq + r;
      SCALAR w = 0.0;
      for (int64_t t = 0; t < L; ++t) w += CONJ(vk[t]) * x[t];
      SCALAR tw = tk * w;
      for (int64_t t = 0; t < L; ++t) x[t] -= tw * vk[t];
    }
  }
  return NULL;
}

int FN(orc_back_transform_)(int64_t n, int64_t b, int64_t nev, const SCALAR *hh_v, const SCALAR *hh_tau,
                            SCALAR *q, int64_t ldq, int nthreads) {
  int64_t K = orc_num_reflectors(n, b, IS_COMPLEX);
  int64_t *r = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
  int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
  orc_reflector_rows(n, b, IS_COMPLEX, r, L);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > nev) nthreads = (int)(nev > 0 ? nev : 1);
  FN(bt_job_t) *jobs = (FN(bt_job_t) *)calloc((size_t)nthreads, sizeof(FN(bt_job_t)));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].n = n;
    jobs[t].b = b;
    jobs[t].K = K;
    jobs[t].c0 = nev * t / nthreads;
    jobs[t].c1 = nev * (t + 1) / nthreads;
    jobs[t].ldq = ldq;
    jobs[t].v = hh_v;
    jobs[t].tau = hh_tau;
    jobs[t].r = r;
    jobs[t].L = L;
    jobs[t].q = q;
  }
  int rc = 0;
  for (int t = 1; t < nthreads; ++t)
    if (pthread_create(&th[t], NULL, FN(bt_worker), &jobs[t]) != 0) rc = -1;
  FN(bt_worker)(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(jobs);
  free(th);
  free(r);
  free(L);
  return rc;
}

/*
 * Full -> band reduction, Eq. 6a (B = P H P^*, Sec. 2.1, Fig. 1), written as
 * its definition: for every column c = 0 .. n-b-1 in turn, one reflector
 * from the column's entries below the band, x = A[c+b : n, c], and the
 * two-sided update A <- H^H A H on the whole dense Hermitian matrix. (A
 * blocked panel algorithm computes the same reflectors: a reflector of
 * column c acts on rows and columns >= c+b, so it never touches the columns
 * of its own panel.) P^* = Q1 = H_0 H_1 ... H_{n-b-1}.
 *
 * a:   in, the full Hermitian matrix (both triangles), n x n column-major.
 *      out, LAPACK-style: entries with |i - j| <= b hold the band matrix B
 *      (the upper triangle the conjugate of the lower), the reflector of column c has v[0] = 1 at row c+b
 *      (implicit) and v[1:] in a[c+b+1 : n, c], the rest of the strictly
 *      upper triangle is zero.
 * tau: out, max(n-b, 0) entries (a length-1 reflector of a real matrix has
 *      tau = 0; of a Hermitian one it makes B[c+b, c] real).
 * Returns the number of reflectors, max(n-b, 0).
 */
int64_t FN(orc_full_to_band_)(int64_t n, int64_t b, SCALAR *a, int64_t lda, SCALAR *tau) {
  int64_t K1 = n > b ? n - b : 0;
  SCALAR *A = (SCALAR *)malloc(sizeof(SCALAR) * (size_t)(n > 0 ? n * n : 1));
  SCALAR *V = (SCALAR *)calloc((size_t)(n > 0 ? n * n : 1), sizeof(SCALAR));
  SCALAR *x = (SCALAR *)malloc(sizeof(SCALAR) * (size_t)(n > 0 ? n : 1));
  SCALAR *v = (SCALAR *)malloc(sizeof(SCALAR) * (size_t)(n > 0 ? n : 1));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) A[i + j * n] = a[i + j * lda];
  for (int64_t c = 0; c < K1; ++c) {
    int64_t r = c + b, L = n - r;
    for (int64_t t = 0; t < L; ++t) x[t] = A[r + t + c * n];
    SCALAR tk;
    double beta;
    FN(house)(L, x, v, &tk, &beta);
    /* left: rows [r, n) of every column, A <- H^H A */
    for (int64_t j = 0; j < n; ++j) {
      SCALAR w = 0.0;
      for (int64_t t = 0; t < L; ++t) w += CONJ(v[t]) * A[r + t + j * n];
      for (int64_t t = 0; t < L; ++t) A[r + t + j * n] -= CONJ(tk) * v[t] * w;
    }
    /* right: columns [r, n) of every row, A <- A H */
    for (int64_t i = 0; i < n; ++i) {
      SCALAR w = 0.0;
      for (int64_t t = 0; t < L; ++t) w += A[i + (r + t) * n] * v[t];
      for (int64_t t = 0; t < L; ++t) A[i + (r + t) * n] -= tk * w * CONJ(v[t]);
    }
    /* column c is beta e_1 below the band, row c its conjugate, exactly */
    A[r + c * n] = beta;
    A[c + r * n] = beta;
    for (int64_t t = 1; t < L; ++t) {
      A[r + t + c * n] = 0.0;
      A[c + (r + t) * n] = 0.0;
    }
    for (int64_t t = 1; t < L; ++t) V[r + t + c * n] = v[t];
    tau[c] = tk;
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      int64_t dlt = i - j;
      if (dlt >= 0 && dlt <= b) /* the lower band; the upper one mirrors it */
        a[i + j * lda] = (i == j) ? RE(A[i + j * n]) : A[i + j * n];
      else if (dlt < 0 && -dlt <= b)
        a[i + j * lda] = CONJ(A[j + i * n]);
      else if (dlt > b)
        a[i + j * lda] = V[i + j * n];
      else
        a[i + j * lda] = 0.0;
    }
  free(A);
  free(V);
  free(x);
  free(v);
  return K1;
}

/*
 * Band -> full back-transformation of eigenvectors, Eq. 6e:
 * C = P^* Y = H_0 H_1 ... H_{K1-1} Y with the reflectors of the full -> band
 * reduction in the layout written by orc_full_to_band (reflector c: v[0] = 1
 * at row c+b, v[1:] = a[c+b+1 : n, c], tau[c]), each applied as in Eq. 8,
 * y <- y - tau v (v^H y), last reflector first. Threads take column blocks.
 */
typedef struct {
  int64_t n, b, K1, c0, c1, lda, ldq;
  const SCALAR *a;
  const SCALAR *tau;
  SCALAR *q;
} FN(bf_job_t);

static void *FN(bf_worker)(void *arg) {
  FN(bf_job_t) *J = (FN(bf_job_t) *)arg;
  for (int64_t k = J->K1 - 1; k >= 0; --k) {
    int64_t r = k + J->b, L = J->n - r;
    const SCALAR *tail = J->a + k * J->lda + r + 1; /* v[1:] */
    SCALAR tk = J->tau[k];
    for (int64_t c = J->c0; c < J->c1; ++c) {
      SCALAR *y = J->q + c * J->ldq + r;
      SCALAR w = y[0];
      for (int64_t t = 1; t < L; ++t) w += CONJ(tail[t - 1]) * y[t];
      SCALAR tauw = tk * w;
      y[0] -= tauw;
      for (int64_t t = 1; t < L; ++t) y[t] -= tauw * tail[t - 1];
    }
  }
  return NULL;
}

int FN(orc_back_transform_full_)(int64_t n, int64_t b, int64_t nev, const SCALAR *a, int64_t lda,
                                 const SCALAR *tau, SCALAR *q, int64_t ldq, int nthreads) {
  int64_t K1 = n > b ? n - b : 0;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > nev) nthreads = (int)(nev > 0 ? nev : 1);
  FN(bf_job_t) *jobs = (FN(bf_job_t) *)calloc((size_t)nthreads, sizeof(FN(bf_job_t)));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].n = n;
    jobs[t].b = b;
    jobs[t].K1 = K1;
    jobs[t].c0 = nev * t / nthreads;
    jobs[t].c1 = nev * (t + 1) / nthreads;
    jobs[t].lda = lda;
    jobs[t].ldq = ldq;
    jobs[t].a = a;
    jobs[t].tau = tau;
    jobs[t].q = q;
  }
  int rc = 0;
  for (int t = 1; t < nthreads; ++t)
    if (pthread_create(&th[t], NULL, FN(bf_worker), &jobs[t]) != 0) rc = -1;
  FN(bf_worker)(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(jobs);
  free(th);
  return rc;
}

#undef FN
#undef CAT
#undef CAT_
