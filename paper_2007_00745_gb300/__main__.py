"""Render one escape-time image to a PPM file, as the paper's program does
(Sec. IV: compute the image, write it, report the computational and the total
time), through the library on cuda:0.

    python -m paper_2007_00745_gb300 --size 8000x8000 --iter-max 2000 --escape-radius 400 \\
        --window -2 1 -1.5 1.5 --sched fcfs_tiles --out Mandelbrot.ppm

Every number comes from the CUDA library; this file only parses arguments and
moves the image to the host.
"""
import argparse
import sys
import time


def parse_size(text):
    """'MxN' -> (rows m, columns n)."""
    try:
        a, b = text.lower().split("x")
        m, n = int(a), int(b)
    except ValueError:
        raise argparse.ArgumentTypeError("size must be ROWSxCOLS, e.g. 480x640")
    if m < 1 or n < 1:
        raise argparse.ArgumentTypeError("size must be positive")
    return m, n


def make_parser():
    p = argparse.ArgumentParser(prog="python -m paper_2007_00745_gb300",
                                description="Render an escape-time (Mandelbrot) image to a PPM file on the GPU.")
    p.add_argument("--size", type=parse_size, default=(480, 640), help="ROWSxCOLS (default 480x640)")
    p.add_argument("--window", type=float, nargs=4, default=[-2.0, 1.0, -1.0, 1.0],
                   metavar=("XMIN", "XMAX", "YMIN", "YMAX"), help="complex window (default -2 1 -1 1)")
    p.add_argument("--iter-max", type=int, default=1000)
    p.add_argument("--escape-radius", type=float, default=2.0, help="escape radius R; the test is |z|^2 > R^2")
    p.add_argument("--sched", default="fcfs_tiles",
                   choices=["naive", "alternating", "fcfs_rows", "fcfs_tiles", "learned"])
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "dfloat"])
    p.add_argument("--cycle-check", action="store_true", help="stop exactly periodic orbits early (same image)")
    p.add_argument("--tile", type=int, default=0)
    p.add_argument("--out", default="Mandelbrot.ppm")
    return p


def main(argv=None):
    args = make_parser().parse_args(argv)
    import torch

    import paper_2007_00745_gb300 as mb

    if not torch.cuda.is_available():
        print("a CUDA device is required", file=sys.stderr)
        return 2
    m, n = args.size
    window = tuple(args.window)
    r2 = args.escape_radius * args.escape_radius
    dev = torch.device("cuda:0")
    out = torch.empty(m * n, dtype=torch.int32, device=dev)
    rgb = torch.empty(m * n * 3, dtype=torch.uint8, device=dev)
    rgb_host = torch.empty(m * n * 3, dtype=torch.uint8, pin_memory=True)
    params = None
    if args.sched == "learned":
        if args.precision != "fp64" or args.cycle_check:
            print("the learned order renders binary64 without cycle detection", file=sys.stderr)
            return 2
        from paper_2007_00745_gb300 import tilemodel
        params, _ = tilemodel.default_model(tile=args.tile or 32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if params is not None:
        mb.mb_render_learned(window, m, n, args.iter_max, r2, out, params, tile=args.tile or 32)
    else:
        mb.mb_render(window, m, n, args.iter_max, r2, out, sched=args.sched, tile=args.tile,
                     precision=args.precision, cycle_check=int(args.cycle_check))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    mb.mb_colorize(out, args.iter_max, rgb)
    rgb_host.copy_(rgb)
    mb.mb_write_ppm(args.out, rgb_host, m, n)
    t2 = time.perf_counter()
    print("computational process time: %.6f s" % (t1 - t0))
    print("total process time: %.6f s" % (t2 - t0))
    print("wrote %s (%d x %d)" % (args.out, n, m))
    return 0


if __name__ == "__main__":
    sys.exit(main())
