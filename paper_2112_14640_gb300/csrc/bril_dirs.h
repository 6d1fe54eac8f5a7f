// bril_dirs.h -- the order and scaling in which the 80 off-centre Brillouin
// links W_s are stored (shared by the builder in links.cu and the stencil in
// brillouin.cuh).
//
// The offsets s in {-1,0,1}^4 \ {0} are grouped by their support
// M = {mu : s_mu != 0} (a 4-bit mask, bit 0 = x ... bit 3 = t), masks in
// increasing order 1..15; inside a group the 2^k sign patterns are numbered by
// b, bit j of b set when the j-th axis of M (in increasing mu) has s_mu = -1.
// Storage index q = group_offset(M) + b.
//
// With k = |s|_1 and lead(M) the highest axis of M (t when s moves in time,
// whose gamma matrix is a plain permutation), the stored matrix is
//   W~_q(n) = rho_k * s_lead * W_s(n),
// which turns the spin factor rho_k sum_mu s_mu gamma_mu - lambda_k/2 of
// Eq. (app_bril) into  sum_mu e_mu gamma_mu - c_k s_lead  with e_mu = s_lead s_mu
// (e_lead = 1) and c_k = lambda_k / (2 rho_k) = 27 * 2^(k-1) / 64.
#pragma once

namespace dgb {
namespace bril {

__host__ __device__ constexpr int popc4(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1); }
__host__ __device__ constexpr int lead_axis(int m) { return (m & 8) ? 3 : (m & 4) ? 2 : (m & 2) ? 1 : 0; }
// number of stored offsets before group M
__host__ __device__ constexpr int group_offset(int m) {
    int o = 0;
    for (int j = 1; j < m; ++j) o += 1 << popc4(j);
    return o;
}
// rho_k = (64, 16, 4, 1) / 432 for k = 1..4
__host__ __device__ constexpr double rho(int k) { return (double)(1 << (2 * (4 - k))) / 432.0; }
// c_k = lambda_k / (2 rho_k), lambda_k = (8, 4, 2, 1) / 64 for k = 1..4
__host__ __device__ constexpr double c_lambda(int k) { return 27.0 / 64.0 * (double)(1 << (k - 1)); }

// storage index and scale of the offset s = (sx, sy, sz, st)
__host__ __device__ inline int store_index(const int s[4], double *scale) {
    int m = 0, b = 0, j = 0;
    for (int mu = 0; mu < 4; ++mu) {
        if (s[mu] == 0) continue;
        m |= 1 << mu;
        if (s[mu] < 0) b |= 1 << j;
        ++j;
    }
    *scale = rho(j) * (double)s[lead_axis(m)];
    return group_offset(m) + b;
}

// W~ memory layout, in complex numbers, of element e of matrix q at site n,
// for either vector layout: (n * 80 + q) * nc^2 + e, one site's 80 matrices
// contiguous in visiting order, so a thread streams its own W~ sequentially.
// (Storing them site-innermost when the vectors are site-inner was measured
// slower: the nine elements of one matrix then sit in nine DRAM pages.)
__host__ __device__ inline long long w_index(int q, int e, long long n, int nc) {
    return (n * 80 + q) * nc * nc + e;
}

}  // namespace bril
}  // namespace dgb
