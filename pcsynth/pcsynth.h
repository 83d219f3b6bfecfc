/* pcsynth.h — seeded synthetic point clouds and camera matrices.
 *
 * This module produces INPUTS only: raw float xyz positions, RGBA8 colours and
 * view-projection matrices. It holds none of the rasterizer's arithmetic (no
 * Morton codes, no batching, no quantization, no projection to pixels), so the
 * GPU library and the CPU oracle can both consume its output without sharing
 * any of the method's code.
 *
 * Every random value is a pure function of (seed, stream, index) through the
 * SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014). Any index range can therefore
 * be generated on its own, in any order and on any number of threads, with the
 * same result.
 *
 * Matrices are 4x4, column-major (m[row + 4*col]), mapping world (x,y,z,1) to
 * OpenGL-style clip coordinates; w_clip = distance along the viewing axis.
 */
#ifndef PCSYNTH_H
#define PCSYNTH_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double extent_m;        /* side of the square area, centred on the origin */
    double wavelength_m;    /* base wavelength of the value noise (octave 0) */
    double amplitude_m;     /* amplitude of octave 0 */
    double persistence;     /* amplitude ratio between octaves */
    double lacunarity;      /* frequency ratio between octaves */
    uint32_t octaves;
    double jitter_m;        /* half-width of the uniform vertical jitter */
    double buildings_frac;  /* fraction of points sampled on box buildings */
    uint32_t n_buildings;
} pcs_terrain_params;

/* Fill `p` with the defaults: 6 octaves, 2 km base wavelength, 300 m amplitude,
 * persistence 0.5, lacunarity 2, 1 cm jitter, no buildings. */
void pcs_terrain_defaults(pcs_terrain_params* p, double extent_m);

/* Points [first, first+n) of the unit-cube cloud: xyz uniform in [0,1)^3 as
 * float, rgba uniform over all 32 bits. xyz has 3*n floats. */
void pcs_unit_cube(uint64_t seed, uint64_t first, uint64_t n,
                   float* xyz, uint32_t* rgba, int threads);

/* Points [first, first+n) of the terrain cloud (plus box buildings when
 * buildings_frac > 0). Colours: height ramp plus noise, alpha 255. */
void pcs_terrain(uint64_t seed, const pcs_terrain_params* p, uint64_t first,
                 uint64_t n, float* xyz, uint32_t* rgba, int threads);

/* Points [first, first+n) of a terrestrial-scan-like terrain cloud in scan
 * order: scan line c = i / points_per_line is a ray from the scanner position
 * (sx, sy) at yaw 2*pi*c/lines (lines = ceil(total / points_per_line)), and
 * its points run outward from 5 m to max_dist_m along it, on the terrain
 * surface; consecutive points therefore form long curves (Sec. 4.2). */
void pcs_terrain_scan(uint64_t seed, const pcs_terrain_params* p, double sx, double sy,
                      double max_dist_m, uint64_t total, uint64_t points_per_line,
                      uint64_t first, uint64_t n, float* xyz, uint32_t* rgba, int threads);

/* Terrain surface height at (x, y), in metres. */
double pcs_terrain_height(uint64_t seed, const pcs_terrain_params* p,
                          double x, double y);

/* Right-handed look-at view followed by an OpenGL perspective projection,
 * computed in double and rounded to float. */
void pcs_look_at_perspective(const double eye[3], const double target[3],
                             const double up[3], double fovy_deg,
                             double aspect, double znear, double zfar,
                             float out[16]);

/* Camera `frame` of an `nframes`-frame seeded fly-through over the terrain:
 * a closed loop at 50-500 m above ground looking ahead and down. Writes the
 * eye position to eye_out when it is not NULL. */
void pcs_flythrough(uint64_t seed, const pcs_terrain_params* p, uint32_t frame,
                    uint32_t nframes, uint32_t width, uint32_t height,
                    float out[16], double eye_out[3]);

/* Oblique overview camera that sees the whole terrain square. */
void pcs_overview(const pcs_terrain_params* p, uint32_t width, uint32_t height,
                  float out[16]);

/* Stereo pair (eye = 0 left, 1 right) of an oblique view over the terrain,
 * eyes separated by ipd_m along the camera's right axis. */
void pcs_stereo(const pcs_terrain_params* p, uint32_t width, uint32_t height,
                double ipd_m, int eye, float out[16]);

/* Seeded random camera around the terrain (for view bundles and serving):
 * eye 50-3000 m above ground inside the area, looking at a random ground
 * point. */
void pcs_random_view(uint64_t seed, const pcs_terrain_params* p, uint64_t index,
                     uint32_t width, uint32_t height, float out[16]);

/* Uniform double in [0,1) for (seed, stream, index); exposed for tests. */
double pcs_uniform(uint64_t seed, uint64_t stream, uint64_t index);

#ifdef __cplusplus
}
#endif
#endif
