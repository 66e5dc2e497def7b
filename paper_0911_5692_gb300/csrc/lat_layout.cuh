// lat_layout.cuh -- how the 7-point step kernel that marches x tiles one warp
// wide (variant 5, lat_xw.cuh) shares the (y tile, z plane) units of one step
// among its block groups. (The 27-point kernel of variant 5 keeps one even
// share of the units in (tile, z) order: with its longer prologue this layout
// measured slower there.)
#pragma once

namespace lat {

// The (y tile, z plane) units of one step, T = N / TY y tiles of zn planes,
// shared among the block groups so that neighbouring y tiles are marched at the
// same planes at the same time: a tile's halo rows are its neighbours' owned
// rows, staged by the neighbouring group moments before, and so come from L2.
// With c = ngroups / T >= 1, the first c T groups take one z chunk of one tile
// each (chunk j of tile t: group j T + t, planes [j zc, (j + 1) zc)); the other
// ngroups - c T groups share the planes [c zc, zn) of every tile in (tile, z)
// order, and zc = T (zn + 2.5) / ngroups gives both kinds the same work with
// about 2.5 planes charged per extra run a shared group starts. With fewer
// groups than tiles all units are shared in (tile, z) order. A group's units
// are [ubeg, uend) of a space of T tiles x zspan planes starting at plane zoff.
struct Layout {
    int ubeg, uend;   // at most (N / TY) N units: 32-bit
    int zspan, zoff;
};

__host__ __device__ __forceinline__ Layout tile_layout(int T, int ngroups, int grp, int zn)
{
    Layout L;
    const int c = ngroups / T;
    const int gt0 = ngroups - c * T;
    if (c < 1 || zn < c + (gt0 > 0 ? 1 : 0)) {   // too few groups, or too few planes for the chunks
        const int U = T * zn;
        L.ubeg = (int)((long long)grp * U / ngroups);
        L.uend = (int)(((long long)grp + 1) * U / ngroups);
        L.zspan = zn;
        L.zoff = 0;
        return L;
    }
    const int gm = c * T, gt = ngroups - gm;
    int zc = gt > 0 ? (int)(((long long)T * (2 * zn + 5)) / (2LL * ngroups)) : (zn + c - 1) / c;
    zc = zc < 1 ? 1 : (zc > zn / c ? zn / c : zc);
    if (gt > 0 && c * zc >= zn) zc = (zn - 1) / c;   // leave the shared groups at least one plane
    if (grp < gm) {
        const int j = grp / T, t = grp - j * T;
        const int zb = j * zc, ze = (gt == 0 && j == c - 1) ? zn : zb + zc;
        L.zspan = ze - zb;
        L.zoff = zb;
        L.ubeg = t * L.zspan;
        L.uend = L.ubeg + L.zspan;
        return L;
    }
    const int zt = zn - c * zc;
    const int U = T * zt;
    const int g = grp - gm;
    L.ubeg = (int)((long long)g * U / gt);
    L.uend = (int)(((long long)g + 1) * U / gt);
    L.zspan = zt;
    L.zoff = c * zc;
    return L;
}

} // namespace lat
