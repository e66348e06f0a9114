// Point order of one tile of the resident engine (host and device).
//
// A block owns its tile [x0, x1) x [y0, y1) and, on every side that has a
// neighbour tile, a ring of width R.  Step s of a block of H iterations updates
// the tile grown by rr = H - s cells (the region R(rr)); its first phase also
// needs ubar one cell further left and below (the region Rp(rr)).  The block's
// points are numbered so that both regions are prefixes of the numbering:
// first the tile (row-major), then frame d = 1 .. R, each frame starting with its
// left/bottom part A_d (bottom row, then left column) and ending with the rest
// B_d (right column, then top row).  With point q owned by thread q mod T, a
// step's active points are then whole warps plus one partial warp.
#pragma once

#ifdef __CUDACC__
#define VOMT_HD __host__ __device__ __forceinline__
#else
#define VOMT_HD inline
#endif

namespace vomt {

struct TileFrame {
    int x0, x1, y0, y1;      // the tile
    int hL, hR, hD, hU;      // 1 where a neighbour tile exists (left, right, below, above)
    int R;                   // ring width (0 for a lone tile)
};

// Points of frame d (1 <= d <= R): in its left/bottom part A_d and in the rest B_d.
VOMT_HD void frame_counts(const TileFrame &f, int d, int &cA, int &cB)
{
    const int TW = f.x1 - f.x0, TH = f.y1 - f.y0;
    const int Wp = TW + (d - 1) * f.hR + d * f.hL;      // bottom row of A_d (and top row of B_d)
    const int Hl = TH + (d - 1) * (f.hU + f.hD);        // left column of A_d
    const int Hr = TH + d * (f.hD + f.hU);              // right column of B_d
    cA = f.hD * Wp + f.hL * Hl;
    cB = f.hR * Hr + f.hU * Wp;
}

// Number of points with ring distance <= d (d = 0: the tile).
VOMT_HD int region_count(const TileFrame &f, int d)
{
    int cnt = (f.x1 - f.x0) * (f.y1 - f.y0);
    for (int j = 1; j <= d && j <= f.R; ++j) {
        int cA, cB;
        frame_counts(f, j, cA, cB);
        cnt += cA + cB;
    }
    return cnt;
}

// Number of points of Rp(rr): R(rr) plus A_{rr+1}.
VOMT_HD int region_p_count(const TileFrame &f, int rr)
{
    int cnt = region_count(f, rr);
    if (rr + 1 <= f.R) {
        int cA, cB;
        frame_counts(f, rr + 1, cA, cB);
        cnt += cA;
    }
    return cnt;
}

// Grid coordinates of point q; false if q is past the last point.
VOMT_HD bool onion_point(const TileFrame &f, int q, int &x, int &y)
{
    const int TW = f.x1 - f.x0, TH = f.y1 - f.y0;
    if (q < 0) return false;
    if (q < TW * TH) {
        x = f.x0 + q % TW;
        y = f.y0 + q / TW;
        return true;
    }
    q -= TW * TH;
    for (int d = 1; d <= f.R; ++d) {
        int cA, cB;
        frame_counts(f, d, cA, cB);
        const int Wp = TW + (d - 1) * f.hR + d * f.hL;
        if (q < cA) {
            if (f.hD && q < Wp) {            // bottom row, left to right
                x = f.x0 - d * f.hL + q;
                y = f.y0 - d;
                return true;
            }
            q -= f.hD * Wp;                  // left column, bottom to top
            x = f.x0 - d;
            y = f.y0 - (d - 1) * f.hD + q;
            return true;
        }
        q -= cA;
        if (q < cB) {
            const int Hr = TH + d * (f.hD + f.hU);
            if (f.hR && q < Hr) {            // right column, bottom to top
                x = f.x1 + d - 1;
                y = f.y0 - d * f.hD + q;
                return true;
            }
            q -= f.hR * Hr;                  // top row, left to right
            x = f.x0 - d * f.hL + q;
            y = f.y1 + d - 1;
            return true;
        }
        q -= cB;
    }
    return false;
}

}  // namespace vomt
