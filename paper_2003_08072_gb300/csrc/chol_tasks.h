// Task list of the one-launch Cholesky sweep (k_ch_dag in k_factor.cu), host code only.
//
// Tasks for nbk diagonal blocks of 32, block step k (the kernel's comment gives the
// operations and the per-tile counters they wait on):
//   F          the whole chain of diagonal blocks (one task, claimed first);
//   T(i,k)     L_ik = A_ik X_kk^T, i >= k + 2;
//   XS(k,j)    X_kj <- X_kk X_kj, j < k;
//   U(i,j,k)   A_ij -= L_ik L_jk^T, k < j <= i, except (k+1, k+1), which F does;
//   XU(i,j,k)  X_ij -= L_ik X_kj, i > k >= j.
// Order: F, then per block step k = 0, 1, ...: the T, the XS, U(k+2, k+1, k) and U(k+2, k+2, k)
// (the tiles F needs at step k + 2), the other U, the XU.  A task is one 32-bit code,
// kind << 27 | i << 18 | j << 9 | k (nbk <= 512).
#pragma once

#include <cstddef>
#include <cstdint>

namespace lpk {

enum : uint32_t { CT_F = 0, CT_T = 1, CT_U = 2, CT_XS = 3, CT_XU = 4 };

inline uint32_t ct_pack(uint32_t kind, int i, int j, int k) {
  return (kind << 27) | ((uint32_t)i << 18) | ((uint32_t)j << 9) | (uint32_t)k;
}

// Writes the codes to out when out is not null; returns their number.
inline size_t chol_dag_tasks(int nbk, uint32_t* out) {
  size_t n = 0;
  auto put = [&](uint32_t kind, int i, int j, int k) {
    if (out) out[n] = ct_pack(kind, i, j, k);
    ++n;
  };
  auto step = [&](int k) {
    for (int i = k + 2; i < nbk; ++i) put(CT_T, i, k, k);
    for (int j = 0; j < k; ++j) put(CT_XS, k, j, k);
    const bool ahead = k + 2 < nbk;   // the two tiles F reads at block step k + 2
    if (ahead) {
      put(CT_U, k + 2, k + 1, k);
      put(CT_U, k + 2, k + 2, k);
    }
    for (int j = k + 1; j < nbk; ++j)
      for (int i = j; i < nbk; ++i) {
        if (i == k + 1 && j == k + 1) continue;
        if (ahead && i == k + 2 && (j == k + 1 || j == k + 2)) continue;
        put(CT_U, i, j, k);
      }
    for (int i = k + 1; i < nbk; ++i)
      for (int j = 0; j <= k; ++j) put(CT_XU, i, j, k);
  };
  put(CT_F, 0, 0, 0);
  for (int k = 0; k < nbk; ++k) step(k);
  return n;
}

}  // namespace lpk
