// The piece schedule of a call that runs in pieces from page-locked host
// buffers: how many pieces, their sizes, and whether each waits for the
// previous one.  Host code only (no CUDA), so that it can be checked on its own.
//
// Two forms.  Staggered: a piece's work waits for the previous piece's
// pre-filter, so that its growth launch queues behind the previous one and
// fills that launch's tail, and pieces end one after another; one piece per
// 2 * pipe_min items (at least 2), equal but for a last one of a quarter.
// Paired: pieces alternate between two streams with no wait, so that two run
// side by side, their sizes falling geometrically to an eighth; at most 4
// pieces.  Calls that
// grow in the 16 x 16 window first take the paired form, the others the
// staggered one.  Calls whose record inputs are copied piece by piece run in two
// equal pieces: the second half's inputs cross the host link while the first
// half is classified.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>

namespace jatam {

constexpr int PIPE_MAX_CHUNKS = 8;

struct PipeSchedule {
    size_t pieces = 0;
    size_t per = 0;  // at least every piece's size: each piece's item list fits a buffer of per items
    size_t sizes[PIPE_MAX_CHUNKS] = {};
    bool stagger = false;  // a piece's work waits for the previous piece's pre-filter
};

// n_items: the call's items, at least 2 * pipe_min.  windowed: the call grows in
// the window first.  staged: its record inputs are copied piece by piece.  form:
// -1 (by the kind of call) or bit 0 staggered, bit 1 geometric sizes.
// pieces_override: 0, or 2 to PIPE_MAX_CHUNKS.  False when the sizes do not add
// up (never for arguments in these ranges).
inline bool pipe_schedule(size_t n_items, size_t pipe_min, bool windowed, bool staged, int form, int pieces_override,
                          PipeSchedule *ps)
{
    PipeSchedule s;
    s.stagger = form >= 0 ? (form & 1) != 0 : !windowed;
    const bool geometric = form >= 0 ? (form & 2) != 0 : windowed;
    size_t pieces = windowed ? std::min(n_items / pipe_min, size_t(4)) : std::max(n_items / (2 * pipe_min), size_t(2));
    if (staged) pieces = 2;
    if (pieces_override) pieces = (size_t)pieces_override;
    pieces = std::min(std::max(pieces, size_t(2)), size_t(PIPE_MAX_CHUNKS));
    size_t left = n_items;
    if (staged) {
        // equal pieces
        s.per = (n_items + pieces - 1) / pieces;
        for (size_t i = 0; i < pieces && left; ++i) {
            s.sizes[i] = std::min(left, s.per);
            left -= s.sizes[i];
        }
    } else if (geometric) {
        // sizes r^i, the last an eighth of the first; the last piece takes the rounding remainder
        const double r = std::pow(0.125, 1.0 / (double)(pieces - 1));
        double tot = 0.0, f = 1.0;
        for (size_t i = 0; i < pieces; ++i, f *= r) tot += f;
        s.per = (size_t)((double)n_items / tot) + 1;
        f = 1.0;
        for (size_t i = 0; i < pieces; ++i, f *= r) {
            size_t m = (i + 1 == pieces) ? left : (size_t)((double)n_items * f / tot);
            m = std::min(std::min(m, left), s.per);
            s.sizes[i] = m;
            left -= m;
        }
    } else {
        // pieces - 1 of per items and a last one of about per / 4: only the last piece's copy is
        // not hidden behind a later piece's classification
        s.per = (size_t)((double)n_items / ((double)pieces - 0.75)) + 1;
        for (size_t i = 0; i < pieces && left; ++i) {
            s.sizes[i] = std::min(left, s.per);
            left -= s.sizes[i];
        }
    }
    size_t used = 0;
    while (used < pieces && s.sizes[used]) ++used;
    s.pieces = used;
    if (left || used == 0) return false;
    for (size_t i = 0; i < used; ++i)
        if (s.sizes[i] > s.per) return false;
    *ps = s;
    return true;
}

}  // namespace jatam
