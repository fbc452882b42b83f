// Host-side check of the z chunks of the EM z-march (zchunk_count,
// zchunk_range, zchunk_of and cell_in_pml_tile from nlf_internal.h) over
// every grid depth, CPML width and chunk length in a range: the chunks tile
// [0, nz) in order without gaps or overlaps, every plane maps back to its
// chunk, interior chunks hold at most kz planes and, with a CPML along z,
// neither they nor their halo planes touch a slab.  Prints the number of
// failures and exits non-zero if there is one.
#include <cstdio>

#include "nlf_internal.h"

using namespace nlf;

int main()
{
    int bad = 0, cases = 0;
    for (int nz = 4; nz <= 300; ++nz)
        for (int cz = 0; cz < 2; ++cz)
            for (int pml = 1; pml <= 16; ++pml)
                for (int kz : {4, 8, 16, 32}) {
                    if (cz && 2 * pml + 4 > nz) continue;       // the C ABI refuses such grids
                    ++cases;
                    const int n = zchunk_count(nz, cz, pml, kz);
                    int next = 0;
                    for (int c = 0; c < n; ++c) {
                        int k0 = 0, k1 = 0;
                        zchunk_range(nz, cz, pml, kz, c, k0, k1);
                        if (k0 != next || k1 <= k0 || k1 > nz) ++bad;
                        for (int k = k0; k < k1; ++k)
                            if (zchunk_of(nz, cz, pml, kz, k) != c) ++bad;
                        const bool interior = !cz || (c > 0 && c < n - 1);
                        if (interior && k1 - k0 > kz) ++bad;
                        if (cz && interior && (k0 - 1 < pml || k1 >= nz - pml)) ++bad;
                        if (cz && !interior && k1 - k0 != pml + 1) ++bad;
                        // a cell of an interior chunk away from the x and y slabs is not in a CPML tile
                        const int n3[3] = {96, 96, nz}, cp[3] = {0, 0, cz};
                        if (interior && cell_in_pml_tile(n3, cp, pml, kz, 40, 40, k0)) ++bad;
                        if (!interior && !cell_in_pml_tile(n3, cp, pml, kz, 40, 40, k0)) ++bad;
                        next = k1;
                    }
                    if (next != nz) ++bad;
                }
    printf("%d cases, %d failures\n", cases, bad);
    return bad != 0;
}
