// Host (FP64) construction of the block Jacobi preconditioner with reverse Cuthill-McKee
// ordering (Section III-D names block Jacobi as the paper's second preconditioner; Section V-G
// applies it after an RCM reordering).
#pragma once

#include <cstdint>
#include <vector>

namespace gmresb3 {

// Reverse Cuthill-McKee order of the symmetric pattern of A + A^T (diagonal excluded):
// components one after another, each started at the unvisited node of smallest degree (ties:
// smallest index) and traversed breadth first with neighbours appended in increasing (degree,
// index) order; the sequence is then reversed.  perm[new] = old.
std::vector<int32_t> rcm_order(int n, const int32_t* rowptr, const int32_t* col);

// Inverses of the diagonal blocks A[I_b, I_b], I_b = perm[b k .. b k + k) (the last block may be
// shorter), by Gauss-Jordan elimination with partial pivoting in FP64; block b's inverse is
// stored column-major at inv[b k k + c k + r] (rows and columns past the block's size are zero).
// Returns false if a block is singular.  Blocks are split over `threads` host threads.
bool block_inverses(int n, const int32_t* rowptr, const int32_t* col, const double* val,
                    const std::vector<int32_t>& perm, int k, std::vector<double>& inv,
                    int threads);

}  // namespace gmresb3
