// lbm_test_encode: the step kernels' 16-bit store codec (round to nearest, or
// stochastic with given random words) applied to pairs of values, so that tests can
// compare it, bit for bit, with independent definitions of the two roundings.
#include "api_common.h"
#include "lbm_device.cuh"

namespace lbm {
namespace codec_test {

// Pair j = (in[2j], in[2j+1]) -> out[j] (low half, high half), unit scale, as a store
// of one 2-field group does it.
template <typename S, bool SR>
__global__ void k_encode_pairs(const float* __restrict__ in, const unsigned* __restrict__ rbits,
                               unsigned* __restrict__ out, long long npair) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= npair) return;
  const float v[2] = {in[2 * j], in[2 * j + 1]};
  const float one[2] = {1.0f, 1.0f};
  if constexpr (SR) out[j] = Codec<S>::enc2_sr(v, one, rbits[j]);
  else out[j] = Codec<S>::enc2(v, one);
}

template <typename S>
void launch(int sround, const float* in, const unsigned* rbits, unsigned* out, long long npair,
            cudaStream_t s) {
  const int block = 256;
  const unsigned grid = (unsigned)((npair + block - 1) / block);
  if (sround) k_encode_pairs<S, true><<<grid, block, 0, s>>>(in, rbits, out, npair);
  else k_encode_pairs<S, false><<<grid, block, 0, s>>>(in, rbits, out, npair);
}

}  // namespace codec_test
}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_test_encode(int store, int stochastic_round, const float* in,
                                      const unsigned* rbits, unsigned* out, long long npair,
                                      void* cuda_stream) {
  if (store != LBM_STORE_F16 && store != LBM_STORE_BF16)
    return fail(LBM_E_INVAL, "store must be LBM_STORE_F16 or LBM_STORE_BF16");
  if (stochastic_round != 0 && stochastic_round != 1)
    return fail(LBM_E_INVAL, "stochastic_round must be 0 or 1");
  if (npair < 0 || npair > (1ll << 30)) return fail(LBM_E_INVAL, "npair must be 0 to 2^30");
  if (npair == 0) return LBM_OK;
  if (!in || !out || (stochastic_round && !rbits)) return fail(LBM_E_INVAL, "NULL buffer");
  const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (store == LBM_STORE_F16) codec_test::launch<__half>(stochastic_round, in, rbits, out, npair, s);
  else codec_test::launch<__nv_bfloat16>(stochastic_round, in, rbits, out, npair, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LBM_E_CUDA, "encode launch failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}
