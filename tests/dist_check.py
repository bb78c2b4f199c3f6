"""Run under torch.distributed.run with 2 ranks (gloo, CPU): bench.py's Dist
helper must give every rank the maximum over ranks and pass its barriers."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from bench import Dist  # noqa: E402


def main():
    d = Dist()
    d.barrier()
    m = d.max(1.5 + d.rank)
    d.barrier()
    print(f"rank {d.rank} world {d.world} max {m}", flush=True)
    d.close()


if __name__ == "__main__":
    main()
