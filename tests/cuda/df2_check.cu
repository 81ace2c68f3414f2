// Test-only CUDA source (built by tests/test_gpu_df2.py, not part of libns3d.so): compares the
// two-lane double-float operations of df2.cuh with the scalar ones of df.cuh bit for bit, lane
// by lane, on pseudo-random inputs generated on the device.  The division and square root of
// df2.cuh take the error term of their last step from the exact product (fma form); their
// scalar references below are written out in that form.
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"
#include "df2.cuh"
#include "k_dir_impl.cuh"

using namespace ns3d;

namespace {

constexpr int NOPS = 16;

__device__ uint64_t mix64(uint64_t z) {  // SplitMix64 finaliser
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// A double-float with |hi| in [2^-40, 2^20), a random sign unless pos, lo of a few ulp(hi) or less.
__device__ df rand_df(uint64_t key, bool pos) {
  const uint64_t r = mix64(key);
  const float m = 1.0f + (float)(r & 0xffffff) * 0x1p-24f;
  const int e = (int)((r >> 24) % 60) - 40;
  float hi = ldexpf(m, e);
  if (!pos && ((r >> 40) & 1)) hi = -hi;
  const float frac = ((float)((r >> 41) & 0xffff) * 0x1p-16f - 0.5f) * 0x1p-23f;
  return df{hi, hi * frac};
}

__device__ bool same(df a, df b) {
  return __float_as_uint(a.hi) == __float_as_uint(b.hi) && __float_as_uint(a.lo) == __float_as_uint(b.lo);
}

// scalar references of df2_div / df2_sqrt (last step in the fma form)
__device__ df ref_div(df x, df y) {
  const float r = rcp_seed(y.hi);
  const float q1 = __fmul_rn(x.hi, r);
  const df p = two_prod(q1, y.hi);
  float rem = __fsub_rn(x.hi, p.hi);
  rem = __fsub_rn(rem, p.lo);
  rem = __fadd_rn(rem, x.lo);
  rem = __fmaf_rn(-q1, y.lo, rem);
  const float s = __fadd_rn(q1, __fmul_rn(rem, r));
  return df{s, __fmaf_rn(rem, r, -__fsub_rn(s, q1))};
}

// scalar reference of df2_offset<false> (the WENO5 offset of the direction pass)
__device__ df ref_offset(df B1, df B2, df B3, df e, df ta, df tb) {
  const df p23 = df_mul_u(B2, B3), p13 = df_mul_u(B1, B3), p12 = df_mul_u(B1, B2);
  const df den = df_add_pos_u(p23, df_add_pos_u(df_mul_f_u(p13, 6.0f), df_mul_f_u(p12, 3.0f)));
  const df num = df_add_fast(df_mul_u(den, e), df_add_fast(df_twice(df_mul_u(p23, ta)), df_mul_f_u(df_mul_u(p12, tb), 3.0f)));
  return ref_div(num, df_mul_f_u(den, 6.0f));
}

// scalar reference of the squared indicators of phase B of the direction pass
__device__ void ref_indicators(df dgm, df dgp, df c133, df eps4, df& B1, df& B2, df& B3) {
  const df ds = df_add_fast(dgp, df_neg(dgm));
  const df s2 = df_sqr_u(ds);
  const df aa = df_add_pos_u(df_mul_u(s2, c133), eps4);
  const df u2 = df_add_fast(dgm, dgp);
  const df b2 = df_add_pos_u(df_sqr_u(u2), aa);
  const df pq = df_add_ordered_u(b2, df_twice(df_twice(s2)));
  const df r4 = df_twice(df_twice(df_mul_u(u2, ds)));
  B1 = df_sqr_u(df_add_ordered(pq, r4));
  B2 = df_sqr_u(b2);
  B3 = df_sqr_u(df_add_ordered(pq, df_neg(r4)));
}
__device__ void new_indicators(df2 dgm, df2 dgp, df2 c133, df2 eps4, df2& B1, df2& B2, df2& B3) {
  const df2 ds = df2_add_fast(dgp, df2_neg(dgm));
  const df2 s2 = df2_sqr_u(ds);
  const df2 aa = df2_add_pos_u(df2_mul_u(s2, c133), eps4);
  const df2 u2 = df2_add_fast(dgm, dgp);
  const df2 b2 = df2_add_pos_u(df2_sqr_u(u2), aa);
  const df2 pq = df2_add_ordered_u(b2, df2_twice(df2_twice(s2)));
  const df2 r4 = df2_twice(df2_twice(df2_mul_u(u2, ds)));
  B1 = df2_sqr_u(df2_add_ordered(pq, r4));
  B2 = df2_sqr_u(b2);
  B3 = df2_sqr_u(df2_add_ordered(pq, df2_neg(r4)));
}

__global__ void k_check(int n, uint64_t seed, int* bad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  df a[2][6];
  for (int l = 0; l < 2; ++l)
    for (int j = 0; j < 6; ++j) a[l][j] = rand_df(seed + 12ull * (uint64_t)t + 6ull * l + j, j >= 2 && j <= 4);
  df2 p[6];
  for (int j = 0; j < 6; ++j) p[j] = df2_pack(a[0][j], a[1][j]);
  const df c133{4.3333335f, -3.9736431e-08f}, eps4{4e-06f, 1e-13f};
  df2 r2[NOPS];
  df r[2][NOPS];
  r2[0] = df2_add_fast(p[0], p[1]);
  r2[1] = df2_add_fast(p[0], df2_neg(p[1]));
  r2[2] = df2_mul_u(p[0], p[1]);
  r2[3] = df2_mul(p[0], p[1]);
  r2[4] = df2_sqr_u(p[0]);
  r2[5] = df2_mul_f_u(p[0], 6.0f);
  r2[6] = df2_add_pos_u(p[2], p[3]);
  r2[7] = df2_add_ordered_u(p[2], p[3]);
  r2[8] = df2_add_ordered(p[2], p[3]);
  r2[9] = df2_twice(p[1]);
  r2[10] = two_prod2(p[0].hi, p[1].hi);
  r2[11] = df2_div(p[0], p[2]);
  r2[12] = df2_offset<false>(p[2], p[3], p[4], p[0], p[1], p[5]);
  new_indicators(p[0], p[1], df2_splat(c133), df2_splat(eps4), r2[13], r2[14], r2[15]);
  for (int l = 0; l < 2; ++l) {
    const df* x = a[l];
    r[l][0] = df_add_fast(x[0], x[1]);
    r[l][1] = df_add_fast(x[0], df_neg(x[1]));
    r[l][2] = df_mul_u(x[0], x[1]);
    r[l][3] = df_mul(x[0], x[1]);
    r[l][4] = df_sqr_u(x[0]);
    r[l][5] = df_mul_f_u(x[0], 6.0f);
    r[l][6] = df_add_pos_u(x[2], x[3]);
    r[l][7] = df_add_ordered_u(x[2], x[3]);
    r[l][8] = df_add_ordered(x[2], x[3]);
    r[l][9] = df_twice(x[1]);
    r[l][10] = two_prod(x[0].hi, x[1].hi);
    r[l][11] = ref_div(x[0], x[2]);
    r[l][12] = ref_offset(x[2], x[3], x[4], x[0], x[1], x[5]);
    ref_indicators(x[0], x[1], c133, eps4, r[l][13], r[l][14], r[l][15]);
  }
  for (int o = 0; o < NOPS; ++o)
    if (!same(df2_lane0(r2[o]), r[0][o]) || !same(df2_lane1(r2[o]), r[1][o])) atomicAdd(&bad[o], 1);
}

}  // namespace

// Runs n lane pairs; bad_host receives NOPS mismatch counts (add_fast, sub, mul_u, mul, sqr_u,
// mul_f_u, add_pos_u, add_ordered_u, add_ordered, twice, two_prod, div, offset, indicator
// B1, B2, B3).  Returns a cudaError_t.
extern "C" int df2_check(int n, unsigned long long seed, int* bad_host) {
  int* bad = nullptr;
  cudaError_t e = cudaMalloc(&bad, sizeof(int) * NOPS);
  if (e != cudaSuccess) return (int)e;
  cudaMemset(bad, 0, sizeof(int) * NOPS);
  k_check<<<(n + 255) / 256, 256>>>(n, seed, bad);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(bad_host, bad, sizeof(int) * NOPS, cudaMemcpyDeviceToHost);
  cudaFree(bad);
  return (int)e;
}

extern "C" int df2_check_nops() { return NOPS; }
