/*
 * CPU oracle for the GEMM kernels -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg may call
 * this.  It shares no code with the CUDA library.
 *
 * Computes, in FP64, the operation the paper's matrix-multiply kernel family
 * evaluates (Section 3: each work item accumulates an R x C output tile from an
 * R x A slice of the left input and an A x C slice of the right input), in its
 * plain definition: one accumulator per output element, k ascending:
 *
 *     C[b,i,j]   = alpha * sum_k op(A)[b,i,k] * op(B)[b,k,j] + beta * C0[b,i,j]
 *     den[b,i,j] = |alpha| * sum_k |op(A)[b,i,k]| * |op(B)[b,k,j]| + |beta| * |C0[b,i,j]|
 *
 * den is the componentwise error scale used to check every GPU result:
 * err = max over entries of |C_gpu - C| / den.  When beta == 0, C0 is not read.
 *
 * Storage is row-major.  op(A) = A (M x K, lda >= K) when transA == 0, and
 * A^T with A stored K x M (lda >= M) when transA == 1; likewise for B.
 * Batch entries are packed with the given element strides.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline double a_at(const double* A, int64_t lda, int transA, int64_t i, int64_t k) {
  return transA ? A[k * lda + i] : A[i * lda + k];
}

static inline double b_at(const double* B, int64_t ldb, int transB, int64_t k, int64_t j) {
  return transB ? B[j * ldb + k] : B[k * ldb + j];
}

static void entry(int transA, int transB, int64_t K, double alpha, const double* A, int64_t lda,
                  const double* B, int64_t ldb, double beta, const double* C0, int64_t ldc,
                  int64_t i, int64_t j, double* c_out, double* den_out) {
  double acc = 0.0, acc_abs = 0.0;
  for (int64_t k = 0; k < K; ++k) {
    double a = a_at(A, lda, transA, i, k);
    double b = b_at(B, ldb, transB, k, j);
    acc += a * b;
    acc_abs += fabs(a) * fabs(b);
  }
  double c0 = (beta != 0.0) ? C0[i * ldc + j] : 0.0;
  *c_out = alpha * acc + beta * c0;
  *den_out = fabs(alpha) * acc_abs + fabs(beta) * fabs(c0);
}

/* Full product.  Outputs C and den are packed (batch, M, N).  nthreads <= 1
 * runs the plain single-thread i-j-k loop; more threads split the rows. */
void oracle_gemm(int transA, int transB, int64_t M, int64_t N, int64_t K, int64_t batch,
                 double alpha, const double* A, int64_t lda, int64_t strideA,
                 const double* B, int64_t ldb, int64_t strideB, double beta,
                 const double* C0, int64_t ldc, int64_t strideC,
                 double* C, double* den, int nthreads) {
  for (int64_t b = 0; b < batch; ++b) {
    const double* Ab = A + b * strideA;
    const double* Bb = B + b * strideB;
    const double* Cb = C0 ? C0 + b * strideC : C0;
    double* Co = C + b * M * N;
    double* Do = den + b * M * N;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
#endif
    for (int64_t i = 0; i < M; ++i)
      for (int64_t j = 0; j < N; ++j)
        entry(transA, transB, K, alpha, Ab, lda, Bb, ldb, beta, Cb, ldc, i, j,
              &Co[i * N + j], &Do[i * N + j]);
  }
}

/* Selected entries only: pos is n triples (b, i, j); outputs are length n. */
void oracle_gemm_entries(int transA, int transB, int64_t K, double alpha,
                         const double* A, int64_t lda, int64_t strideA,
                         const double* B, int64_t ldb, int64_t strideB, double beta,
                         const double* C0, int64_t ldc, int64_t strideC,
                         int64_t n, const int64_t* pos, double* C, double* den, int nthreads) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
#endif
  for (int64_t s = 0; s < n; ++s) {
    int64_t b = pos[3 * s], i = pos[3 * s + 1], j = pos[3 * s + 2];
    entry(transA, transB, K, alpha, A + b * strideA, lda, B + b * strideB, ldb, beta,
          C0 ? C0 + b * strideC : C0, ldc, i, j, &C[s], &den[s]);
  }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
