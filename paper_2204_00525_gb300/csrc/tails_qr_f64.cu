// Instantiation of the fused tails + register QR leaf for float64, and the dispatch of
// both precisions on the block's padded column count.
#include "tails_qr.cuh"

namespace fig {

void tails_qr_f32(const LeafParams& p, int nreg, int n, double* tri_out, cudaStream_t st);

static void tails_qr_f64(const LeafParams& p, int nreg, int n, double* tri_out, cudaStream_t st) {
  switch (nreg) {
    case 2: launch_tails_qr<double, 2>(p, n, tri_out, st); break;
    case 4: launch_tails_qr<double, 4>(p, n, tri_out, st); break;
    case 6: launch_tails_qr<double, 6>(p, n, tri_out, st); break;
    case 8: launch_tails_qr<double, 8>(p, n, tri_out, st); break;
    case 10: launch_tails_qr<double, 10>(p, n, tri_out, st); break;
    case 12: launch_tails_qr<double, 12>(p, n, tri_out, st); break;
    case 14: launch_tails_qr<double, 14>(p, n, tri_out, st); break;
    case 16: launch_tails_qr<double, 16>(p, n, tri_out, st); break;
    case 20: launch_tails_qr<double, 20>(p, n, tri_out, st); break;
    case 24: launch_tails_qr<double, 24>(p, n, tri_out, st); break;
    case 28: launch_tails_qr<double, 28>(p, n, tri_out, st); break;
    default: launch_tails_qr<double, 32>(p, n, tri_out, st); break;
  }
}

void tails_qr(const LeafParams& p, const TsqrBlock& b, cudaStream_t st, int64_t* launches) {
  if (p.N == 0 || p.n_tiles == 0) return;
  if (p.mixed) tails_qr_f32(p, b.nreg, b.n, b.tri[0], st);
  else tails_qr_f64(p, b.nreg, b.n, b.tri[0], st);
  ++*launches;
}

}  // namespace fig
