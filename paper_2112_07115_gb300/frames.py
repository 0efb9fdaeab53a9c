"""Runs frames of one workload through the C ABI, for profilers (ncu) and
quick checks: python -m paper_2112_07115_gb300.frames --workload toy
--mode coherent --frames 10. Prints one line of frame statistics per frame.

Workloads: toy (the toy street, 10k rays, 3 reflections), highway (1M rays,
4 reflections, 200 roof receivers; --freq selects 28 or 5.9 GHz), roadside
(the highway with 200 static roadside receivers), city (8 x 8 box buildings).
--diffraction-order turns diffraction on (up to that many wedges),
--diffraction-reflections adds reflections around it."""
import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", choices=["toy", "highway", "roadside", "city"], default="toy")
    ap.add_argument("--mode", choices=["full", "coherent"], default="coherent")
    ap.add_argument("--frames", type=int, default=10)
    ap.add_argument("--freq", type=float, default=28e9)
    ap.add_argument("--rays", type=int, default=0, help="ray count (0: the workload's own)")
    ap.add_argument("--diffraction-order", type=int, default=0, help="0: no diffraction, else 1-3")
    ap.add_argument("--diffraction-reflections", type=int, default=0,
                    help="with diffraction: reflections around it (0-3)")
    args = ap.parse_args(argv)

    import torch
    from paper_2112_07115_gb300 import build, dcem, scenes
    build.build()
    torch.cuda.set_device(0)
    n = args.frames + 1
    if args.workload == "toy":
        sc = scenes.toy_street()
    elif args.workload == "highway":
        sc = scenes.highway(seed=0, n_frames=n, n_rays=args.rays or 1_000_000, max_refl=4, freq_hz=args.freq)
    elif args.workload == "roadside":
        sc = scenes.highway(seed=0, n_frames=n, n_rays=args.rays or 1_000_000, max_refl=4, freq_hz=args.freq,
                            roadside_rx=200)
    else:
        sc = scenes.city_blocks(n_rays=args.rays or 200_000, freq_hz=args.freq)
    n_rays = args.rays or sc.n_rays
    s = dcem.Scene.from_scene(sc, stream=torch.cuda.current_stream().cuda_stream)
    s.set_rays(scenes.fibonacci_sphere(n_rays))
    if args.diffraction_order:
        s.set_diffraction(True)
        s.set_diffraction_order(args.diffraction_order)
        if args.diffraction_reflections:
            s.set_diffraction_reflections(args.diffraction_reflections)
    mode = dcem.MODE_COHERENT if args.mode == "coherent" else dcem.MODE_FULL
    prm = dcem.default_params(max_refl=sc.max_refl, freq_hz=sc.freq_hz, mode=mode)
    for i in range(args.frames):
        f = i % sc.nframes
        if sc.nobj:
            s.update_transforms(sc.xf[f])
        fr = s.trace(sc.tx, sc.rx[f], prm)
        st = fr.stats
        print(f"frame {i}: coherent {st['coherent']} segments {st['segments_traced']} "
              f"retraced {st['rays_retraced']} keys {st['unique_candidates']} reused {st['keys_reused']} "
              f"paths {st['paths_valid']}", flush=True)
    s.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
