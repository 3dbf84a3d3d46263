// strip_oracle.cpp -- TEST INFRASTRUCTURE ONLY: plain reference of the strip
// clustering of Sec. 4 (Towards an HLT implementation), one module after the
// other, one strip after the other, in the order the section describes it:
//  * a seed strip has ADC above 3 times its expected noise;
//  * a cluster adds to its seeds every strip above twice the noise that is
//    consecutive, or separated by a small gap; the gap's allowed size depends
//    on bad strips (reading: only bad strips can be bridged, at most
//    max_bad_gap of them in a row; a bad strip carries no charge and no noise);
//  * the cluster is kept if the quadrature sum of its ADCs exceeds 5 times the
//    quadrature sum of its noises and its total charge reaches q_min.
// Noise comes in eighths of an ADC count (noise_q = 8 noise), so every test is
// an exact integer comparison: 8 a > 3 nq, 8 a > 2 nq, 64 sum a^2 > 25 sum nq^2.
// Shares no code with the CUDA library.
#include <cstdint>

extern "C" int orc_strip_clusters(int n_modules, int n_strips, const uint16_t* adc, const uint16_t* noise_q,
                                  const uint8_t* bad, int max_bad_gap, int q_min, int max_out, int* out_module,
                                  int* out_first, int* out_last, int* out_charge, double* out_center) {
  int n_out = 0;
  for (int m = 0; m < n_modules; ++m) {
    const uint16_t* a = adc + (int64_t)m * n_strips;
    const uint16_t* nq = noise_q + (int64_t)m * n_strips;
    const uint8_t* b = bad + (int64_t)m * n_strips;
    bool open = false, seeded = false;
    int first = 0, last = 0, pending_bad = 0;
    int64_t q = 0, q2 = 0, n2 = 0, qi = 0;
    auto close = [&]() {
      if (open && seeded && 64 * q2 > 25 * n2 && q >= q_min) {
        if (n_out < max_out) {
          out_module[n_out] = m;
          out_first[n_out] = first;
          out_last[n_out] = last;
          out_charge[n_out] = (int)q;
          out_center[n_out] = (double)qi / (double)q;
        }
        ++n_out;
      }
      open = false;
      seeded = false;
      pending_bad = 0;
    };
    for (int i = 0; i < n_strips; ++i) {
      if (b[i]) {
        if (open && ++pending_bad > max_bad_gap) close();
        continue;
      }
      const int64_t ai = a[i], ni = nq[i];
      if (8 * ai > 2 * ni) {
        if (!open) {
          open = true;
          first = i;
          q = q2 = n2 = qi = 0;
        }
        last = i;
        pending_bad = 0;
        q += ai;
        q2 += ai * ai;
        n2 += ni * ni;
        qi += (int64_t)i * ai;
        if (8 * ai > 3 * ni) seeded = true;
      } else {
        close();
      }
    }
    close();
  }
  return n_out;
}
