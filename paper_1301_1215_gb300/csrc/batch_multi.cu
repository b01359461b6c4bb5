// The multi-side pass kernels of batches (kernels.cuh, "batches of several sides"): every pass mode, generic and
// standard-field-of-view forms, with the dynamic shared memory each needs for its largest side.
#include <algorithm>

#include "kernels.cuh"

namespace nlv {

namespace {

template <int N1, int N2> void side_smem(MultiKernels& m) {
  using S = Split<N1, N2>;
  constexpr int lanes = kRowMaxThreads / S::TL;
  for (int mode = 0; mode < NUM_ROW_MODES; ++mode)
    m.row_smem[mode] = std::max(m.row_smem[mode], row_smem(mode, S::N, lanes, S::SM_LANE).total);
  for (int mode = 0; mode < NUM_COL_MODES; ++mode)
    m.col_smem[mode] =
        std::max(m.col_smem[mode], col_smem(mode, S::N, NLV_COL_C, S::SM_LANE_COL, S::N / 2).total);
}

MultiKernels make_multi() {
  MultiKernels m{};
  m.row[ROW_W_IFFT] = (const void*)row_pass_multi<ROW_W_IFFT, false>;
  m.row[ROW_PSF] = (const void*)row_pass_multi<ROW_PSF, false>;
  m.row[ROW_FFT_P_OUT] = (const void*)row_pass_multi<ROW_FFT_P_OUT, false>;
  m.row[ROW_FFT_RESID] = (const void*)row_pass_multi<ROW_FFT_RESID, false>;
  m.row[ROW_P_IFFT] = (const void*)row_pass_multi<ROW_P_IFFT, false>;
  m.row[ROW_FFT_W_ADJ] = (const void*)row_pass_multi<ROW_FFT_W_ADJ, false>;
  m.row[ROW_FFT_W_NORMAL] = (const void*)row_pass_multi<ROW_FFT_W_NORMAL, false>;
  m.row[ROW_FFT_W_RHS] = (const void*)row_pass_multi<ROW_FFT_W_RHS, false>;
  m.col[COL_IFFT_C] = (const void*)col_pass_multi<COL_IFFT_C, false>;
  m.col[COL_PROD_FFT] = (const void*)col_pass_multi<COL_PROD_FFT, false>;
  m.col[COL_SIM_FFT] = (const void*)col_pass_multi<COL_SIM_FFT, false>;
  m.col[COL_IFFT_PROD_FFT] = (const void*)col_pass_multi<COL_IFFT_PROD_FFT, false>;
  m.col[COL_IFFT_ADJ_FFT] = (const void*)col_pass_multi<COL_IFFT_ADJ_FFT, false>;
  m.row_std[ROW_W_IFFT] = (const void*)row_pass_multi<ROW_W_IFFT, true>;
  m.row_std[ROW_PSF] = (const void*)row_pass_multi<ROW_PSF, true>;
  m.row_std[ROW_FFT_W_NORMAL] = (const void*)row_pass_multi<ROW_FFT_W_NORMAL, true>;
  m.col_std[COL_IFFT_PROD_FFT] = (const void*)col_pass_multi<COL_IFFT_PROD_FFT, true>;
  side_smem<8, 16>(m);
  side_smem<12, 16>(m);
  side_smem<16, 16>(m);
  side_smem<16, 20>(m);
  side_smem<16, 24>(m);
  return m;
}

}  // namespace

const MultiKernels* multi_kernels() {
  static const MultiKernels m = make_multi();
  return &m;
}

}  // namespace nlv
