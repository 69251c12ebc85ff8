// k_halo.cu -- halo strips of a lattice split into slabs along the periodic
// direction q^2.
//
// The update (Eq. 12) pulls population a of cell (i, j) from (i - c1, j - c2),
// so a slab's first columns read, for every population with c2 > 0, the
// c2 columns before it, and its last columns, for c2 < 0, the |c2| columns
// after it: D2Q21 needs 7 populations at depth 1, 4 at depth 2 and 1 at
// depth 3 on each side (12 strips), D2Q9 3 at depth 1.  A strip covers every
// stored row, the ghost rows of the walls included (App. B fills them per
// column, so a neighbour's ghost rows are this slab's).  Values move as
// stored (deviations in the storage type), bit for bit.
#include "clbm_internal.cuh"

namespace clbm {

namespace {

// Entry e of the strips whose populations have c2 of the given sign:
// populations in ascending order, depths 1 .. |c2| within each.  Returns
// false past the last entry.
__host__ __device__ inline bool halo_entry(int Q, int sign, int e, int* a_out, int* d_out) {
    int k = 0;
    for (int a = 1; a < Q; ++a) {
        const int c2 = c2_of(a);
        if (c2 * sign <= 0) continue;
        const int depth = c2 > 0 ? c2 : -c2;
        for (int d = 1; d <= depth; ++d, ++k)
            if (k == e) {
                *a_out = a;
                *d_out = d;
                return true;
            }
    }
    return false;
}

// One thread per (entry, stored row).  side 0: the strips the lower
// neighbour (columns before this slab) needs, or, unpacking, the strips it
// sends; side 1 likewise for the upper neighbour.  Packing copies interior
// columns, unpacking writes ghost columns (storage column = interior + GC).
template <typename W>
__global__ void k_halo(W* __restrict__ state, W* __restrict__ buf, int Q, long long plane, int ld,
                       int rows, int n2, int side, int unpack, int nent) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = blockIdx.y;
    if (row >= rows || e >= nent) return;
    // packing for the lower neighbour sends c2 < 0; receiving from it takes c2 > 0
    const int sign = (side == 0) == (unpack != 0) ? 1 : -1;
    int a = 0, d = 0;
    if (!halo_entry(Q, sign, e, &a, &d)) return;
    int col;
    if (!unpack) col = side == 0 ? d - 1 : n2 - d;       // interior columns sent
    else col = side == 0 ? -d : n2 + d - 1;             // ghost columns received
    W* p = state + a * plane + (long long)row * ld + col + GC;
    W* q = buf + (long long)e * rows + row;
    if (unpack) *p = *q;
    else *q = *p;
}

}  // namespace

int halo_entries(int Q) {
    int n = 0, a, d;
    while (halo_entry(Q, 1, n, &a, &d)) ++n;
    return n;
}

void launch_halo(int Q, int prec, void* state, void* buf, long long plane, int ld, int rows, int n2,
                 int side, int unpack, cudaStream_t stream) {
    const int nent = halo_entries(Q);
    const dim3 grid((rows + 127) / 128, nent);
    switch (storage_bytes(prec)) {
        case 8:
            k_halo<unsigned long long><<<grid, 128, 0, stream>>>((unsigned long long*)state,
                                                                 (unsigned long long*)buf, Q, plane, ld,
                                                                 rows, n2, side, unpack, nent);
            break;
        case 4:
            k_halo<unsigned><<<grid, 128, 0, stream>>>((unsigned*)state, (unsigned*)buf, Q, plane, ld, rows,
                                                       n2, side, unpack, nent);
            break;
        default:
            k_halo<unsigned short><<<grid, 128, 0, stream>>>((unsigned short*)state, (unsigned short*)buf, Q,
                                                             plane, ld, rows, n2, side, unpack, nent);
    }
}

}  // namespace clbm
