// bounds.h - the predicate behind the debug build's device-side neighbour-index checks.
//
// The kernels compute every neighbour from the site's coordinates (no tables); in the library's
// debug build (compiled with LQCD_DEBUG_BOUNDS) each computed neighbour address is tested with
// lqcd_neighbour_ok before it is used.  A failing test sets a bit of the context's error word
// (lqcd_bounds_word) and the hop reads site 0 instead, so the kernel never touches memory outside
// its buffers and never traps.  Plain integer code, usable on the host (the CPU tests call it) and
// on the device.
#pragma once

#ifdef __CUDACC__
#define LQCD_HD __host__ __device__
#else
#define LQCD_HD
#endif

// error-word bits
#define LQCD_BOUNDS_NEIGHBOUR 1u  // a neighbour address outside [0, V)

// true when l is a site address of a lattice with vh sites per parity, i.e. 0 <= l < 2 vh (so that
// its half-lattice index l >> 1 lies in [0, vh))
LQCD_HD inline bool lqcd_neighbour_ok(long long l, long long vh) { return vh > 0 && l >= 0 && l < 2 * vh; }
