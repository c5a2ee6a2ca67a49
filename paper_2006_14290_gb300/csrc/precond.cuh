// Block-Jacobi preconditioner setup (the Jacobi setup is declared with the
// SpMV entry points).
#pragma once
#include "spmv.cuh"

namespace gko {

// B[i*bs + j] = row i of the inverse of its diagonal block (blocks of bs
// rows, the last one n % bs rows when bs does not divide n) at column j,
// zeros past a short block; A: an FP64 CSR matrix.  singular (device
// counter, nullable) counts the blocks left unscaled.
constexpr int kBlockJacobiMax = 32;
int block_jacobi_inverse(const gko_matrix_s* A, int bs, double* B, unsigned long long* singular, cudaStream_t s);

}  // namespace gko
