"""Regenerate csrc/generated/*.cuh:  python -m paper_2510_05100_b300.codegen"""
import os

from .qcd_bg import emit_all

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "generated", "qcd_amplitudes.cuh")


def generate(path: str = OUT) -> bool:
    """Write the generated header; return True if its content changed."""
    text = emit_all()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as f:
            f.write(text)
        return True
    return False


if __name__ == "__main__":
    changed = generate()
    print(("wrote " if changed else "unchanged ") + OUT)
