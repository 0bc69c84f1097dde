/*
 * csr_omp.c -- the oracle's sparse matrix-vector product y = A x over the rows
 * of a CSR matrix, split across OpenMP threads.
 *
 * TEST INFRASTRUCTURE ONLY (part of the CPU oracle; see fe_oracle.py).  Each
 * row is summed in column order by one thread, exactly the textbook CSR
 * product; threads only divide the rows.  It lets the oracle's solves use the
 * host's cores, as scipy's CSR product runs on one thread.
 */
#include <stdint.h>

void oracle_csr_matvec(int64_t n_rows, const int64_t* indptr, const int32_t* indices, const double* data,
                       const double* x, double* y, int nthreads) {
#pragma omp parallel for schedule(static) num_threads(nthreads)
  for (int64_t i = 0; i < n_rows; ++i) {
    double s = 0.0;
    for (int64_t k = indptr[i]; k < indptr[i + 1]; ++k) s += data[k] * x[indices[k]];
    y[i] = s;
  }
}
