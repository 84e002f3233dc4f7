// Register-window tile application shared by the real back-transformation
// kernels (wavefront and pipeline variants).
#pragma once

namespace gb {

// Apply one tile: the nb reflectors staged in vs/ts, sweep offset q = nb-1
// down to 0 (descending sweep = reverse generation order), to the window w
// of one column.  Reflector q covers window rows q .. q+B-1; vs[q][0] is the
// implicit 1 and vs[q][i] = 0 past the reflector's length, so truncated
// reflectors need no special case.  Per reflector: B-1 DFMA for the dot
// product (the v_0 term is the initial value), one DMUL for tau*w, one DADD
// and B-1 DFMA for the update: 2*B FP64 operations, the algorithmic count.
template <int B, int NB>
__device__ __forceinline__ void apply_tile_regs(double (&w)[B + NB - 1], const double (*vs)[B],
                                                const double *ts)
{
#pragma unroll
    for (int q = NB - 1; q >= 0; q--) {
        const double tau = ts[q];
        if (tau != 0.0) {
            double acc = w[q];
#pragma unroll
            for (int i = 1; i < B; i++) acc = fma(vs[q][i], w[q + i], acc);
            const double tw = tau * acc;
            w[q] -= tw;
            // Re-read v from shared memory instead of keeping B values live
            // across both loops (the window already holds B+NB-1 registers).
            const volatile double *vq = vs[q];
#pragma unroll
            for (int i = 1; i < B; i++) w[q + i] = fma(-tw, vq[i], w[q + i]);
        }
    }
}

}  // namespace gb
