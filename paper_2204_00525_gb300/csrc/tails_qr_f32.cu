// Instantiation of the fused tails + register QR leaf for the mixed path (float tiles).
#include "tails_qr.cuh"

namespace fig {

void tails_qr_f32(const LeafParams& p, int nreg, int n, double* tri_out, cudaStream_t st) {
  switch (nreg) {
    case 2: launch_tails_qr<float, 2>(p, n, tri_out, st); break;
    case 4: launch_tails_qr<float, 4>(p, n, tri_out, st); break;
    case 6: launch_tails_qr<float, 6>(p, n, tri_out, st); break;
    case 8: launch_tails_qr<float, 8>(p, n, tri_out, st); break;
    case 10: launch_tails_qr<float, 10>(p, n, tri_out, st); break;
    case 12: launch_tails_qr<float, 12>(p, n, tri_out, st); break;
    case 14: launch_tails_qr<float, 14>(p, n, tri_out, st); break;
    case 16: launch_tails_qr<float, 16>(p, n, tri_out, st); break;
    case 20: launch_tails_qr<float, 20>(p, n, tri_out, st); break;
    case 24: launch_tails_qr<float, 24>(p, n, tri_out, st); break;
    case 28: launch_tails_qr<float, 28>(p, n, tri_out, st); break;
    default: launch_tails_qr<float, 32>(p, n, tri_out, st); break;
  }
}

}  // namespace fig
