// Launch of the adaptive k-NN query kernel (search_kernel.cuh): the launch
// shape -- positions per lane per streaming step, warps per query and CTAs per
// SM -- picks one of the instantiations compiled in kernels_search_u*w*.cu.
#include "search_kernel.cuh"

namespace pf {

namespace {

using skern::Dev;
using skern::cand_buf;

// q | runs | ranges | qsk | cpre | ppre | top-k | warp lists | warp candidate buffers
size_t search_smem(int d_pad, int L, int M, int k_max, int U, int QW) {
  return size_t(d_pad) * 4 + size_t(L) * 24 + size_t(M) * 8 + size_t(L + 1) * 8 + size_t(k_max) * 8 * (1 + QW) +
         size_t(cand_buf(U)) * 4 * QW;
}

// 8 warps per query only with 8 positions per lane; a shape with flat_fill > 0
// takes the instantiation that can stream rounds flat
skern::Kernel pick_search_kernel(int d_pad, int U, int QW, bool flat) {
  if (QW == 8) return flat ? skern::pick_u8w8_flat(d_pad) : skern::pick_u8w8(d_pad);
  if (U == 4) return flat ? skern::pick_u4w4_flat(d_pad) : skern::pick_u4w4(d_pad);
  return flat ? skern::pick_u8w4_flat(d_pad) : skern::pick_u8w4(d_pad);
}

}  // namespace

cudaError_t launch_search(const pf_index* ix, const SearchArgs& a, cudaStream_t s) {
  if (a.Q <= 0) return cudaSuccess;
  Dev P;
  P.n = int(ix->n);
  P.d = ix->d;
  P.d_pad = ix->lay.d_pad;
  P.L = ix->L;
  P.Kb = ix->lay.Kb;
  P.M = ix->M;
  P.B = ix->B;
  P.family = ix->family;
  P.ell = ix->lay.ell;
  P.x32 = ix->x32;
  P.xf16 = ix->xf16;
  P.x16 = ix->x16;
  P.x8 = ix->x8;
  P.x8_meta = ix->x8_meta;
  P.codes = ix->codes;
  P.ids = ix->ids;
  P.pfx = ix->pfx;
  P.sk = ix->sk;
  P.skc = ix->skc;
  P.cpP = ix->cpP;
  P.cos_tab = a.cos_tab ? a.cos_tab : ix->cos_tab;
  P.bf16_err = ix->bf16_err;
  P.Q = a.Q;
  P.qx = a.qx;
  P.qcodes = a.qcodes;
  P.qsk = a.qsk;
  P.k = a.k;
  P.recall = a.recall;
  P.start = a.start;
  P.k_max = a.k_max;
  P.filter = a.filter;
  P.scoring = a.scoring;
  P.out_ids = a.out_ids;
  P.out_sims = a.out_sims;
  P.stats = a.stats;
  P.counter = a.counter;
  P.path_count = ix->path_count;
  P.stop_every = a.stop_every;
  P.pool_fns = ix->pool_fns;
  P.pool_rule = a.pool_rule;
  const SearchShape sh = a.shape.unroll ? a.shape : ix->search_shape;
  P.flat_fill = sh.flat_fill;
  const int U = sh.unroll == 4 ? 4 : 8, QW = sh.warps == 8 ? 8 : 4;
  const size_t smem = search_smem(P.d_pad, P.L, P.M, P.k_max, U, QW);
  skern::Kernel kern = pick_search_kernel(P.d_pad, U, QW, sh.flat_fill > 0);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * QW, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (sh.ctas_per_sm > 0 && sh.ctas_per_sm < per_sm) per_sm = sh.ctas_per_sm;
  int blocks = ix->num_sms * per_sm;
  if (blocks > a.Q) blocks = a.Q;
  kern<<<blocks, 32 * QW, smem, s>>>(P);
  return cudaGetLastError();
}

int search_max_ctas_per_sm(const pf_index* ix, int k_max, int unroll, int warps) {
  const int U = unroll == 4 ? 4 : 8, QW = warps == 8 ? 8 : 4;
  const size_t smem = search_smem(ix->lay.d_pad, ix->L, ix->M, k_max, U, QW);
  skern::Kernel kern = pick_search_kernel(ix->lay.d_pad, U, QW, false);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * QW, smem) != cudaSuccess) return 0;
  return per_sm;
}

}  // namespace pf
