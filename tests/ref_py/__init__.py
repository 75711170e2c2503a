"""Independent pure-Python transcription of HighwayHash (test infrastructure)."""
